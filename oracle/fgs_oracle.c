/*
 * fgs_oracle.c - plain FP64 CPU oracle of the Fisheye-GS hot path
 * (Fisheye-GS: equidistant-fisheye 3D Gaussian splatting, arXiv 2409.04751).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the benchmark's
 * cpu_baseline / reference leg load this library. The product (CUDA) path never calls it and
 * shares no code, header, table or constant with it.
 *
 * What it computes, step by step, with the passage each step follows:
 *   orc_project     per Gaussian: view transform (Sec. 3.1 "Transformation"), equidistant
 *                   projection of the mean (Sec. 3.2, eq. "equal_distance" and the x_p, y_p
 *                   equations; other models below), fisheye Jacobian J_phi (Sec. 4.2),
 *                   Sigma = R S S^T R^T
 *                   (Sec. 3.1 "Definition"), Sigma_p = T Sigma T^T with T = J W (Sec. 4.3),
 *                   conic, colour from spherical harmonics, depth, footprint.
 *   orc_render      per pixel: the blending sum of Sec. 3.1 "Rendering" evaluated over every
 *                   Gaussian whose alpha reaches 1/255 at that pixel, in depth order.
 *   orc_backward    gradients of L = sum_p <dL/dC_p, C_p>: the per-pixel blend derivative,
 *                   then dmu_c = J^T dmu_p (Sec. 4.2 backward), dJ/d{x_c,y_c,z_c} with
 *                   S1..S8 (Sec. 4.3 backward), the accumulation of both on mu (end of
 *                   Sec. 4.3), and Sigma -> (s, q), colour -> SH and view direction.
 *   orc_build_keys  tile binning and sort (Sec. 3.1 "Rendering", Sec. 4.1): one
 *                   (tile << 32 | depth bits) key per Gaussian x covered tile, stable order;
 *                   optionally only the tiles the alpha >= 1/255 ellipse reaches (the precise
 *                   Gaussian-tile intersection of the renderers of Sec. 6 / Table 3).
 *
 * Camera models (camera[18]): 0 the equidistant fisheye of the method; 1 equisolid,
 * 2 stereographic, 3 orthographic, the other radial models Sec. 3.2 names (r_d = f r(theta)
 * with r = 2 sin(theta/2), 2 tan(theta/2), sin(theta)); 5 the pinhole camera the method is
 * compared with (r = tan(theta): x_p = cx + fx x_c / z_c); 4 the equirectangular panorama of the
 * "Extension to Other Camera Models" paragraph (Sec. 6): x_p = cx + fx atan2(x_c, z_c),
 * y_p = cy + fy atan2(y_c, sqrt(x_c^2 + z_c^2)), which with fx = w / 2 pi, cx = w / 2,
 * fy = h / pi, cy = h / 2 is the paper's pair of equations.
 *
 * Readings where the paper is silent or garbled (each is a convention, "parity unpinned" as a
 * constant: the paper fixes none of the numbers below):
 *   - theta = atan2(l_z, z_c) in [0, pi]; the printed arctan(l_z / z_c) is wrong for z_c < 0.
 *   - J_phi as printed lacks f_x, f_y on its theta terms; the oracle uses the exact derivative
 *       J = [[fx (g + x^2 h), fx x y h, -fx x / l2], [fy x y h, fy (g + y^2 h), -fy y / l2]],
 *     g = theta / l_z, h = (z l_z / l2 - theta) / l_z^3, l2 = |mu_c|^2 (printed: "of mu_p").
 *   - dJ/dy_c entry [0, 2] is printed as 2 fy x y / l2^2; the exact value is 2 fx x y / l2^2.
 *   - Near the optical axis the quotients h = S7 / (l2^2 l_z^5) and S8 / (l2^2 l_z^5) lose
 *     all digits to cancellation; for t = l_z / z_c < 1e-2 they are evaluated by their Taylor
 *     series in t (derived from atan's series), which is exact to rounding there.
 *   - camera axes x right, y down, z forward; pixel (i, j) is sampled at (i + 0.5, j + 0.5).
 *   - a Gaussian is visible iff |mu_c| > 0.2, theta < pi - 0.05 and opacity >= 1/255;
 *     orthographic and pinhole: theta < pi/2 - 0.05 (beyond it r(theta) decreases, or does
 *     not exist); the pinhole also culls a Gaussian whose projected mean lies outside the
 *     guard band |x_p - c_x| <= 1.3 W/2, |y_p - c_y| <= 1.3 H/2 (the 1.3 tan(FOV/2) limit of
 *     the pinhole renderer the method is compared with, applied as a cull: outside it the
 *     affine footprint of a Gaussian grazing the image is ill-conditioned);
 *     panorama: |latitude| < pi/2 - 0.05 (the poles, where J is singular). The panorama has no
 *     wrap-around at longitude +-pi: a Gaussian is drawn on the side of its mean only.
 *   - every radial model's Jacobian has the form of the equidistant one,
 *       J = [[fx (g + x^2 h), fx x y h, fx x k], [fy x y h, fy (g + y^2 h), fy y k]],
 *     g = r(theta) / l_z, h = (1/l) dG/dl, k = dG/dz + z h for g = G(l, z), l = |mu_c|
 *     (equidistant: k = -1 / l2).
 *   - Sigma_p gets 0.3 added on its diagonal (low-pass dilation of the renderer the method
 *     plugs into).
 *   - colour = max(0, sum_k SH_k Y_k(dir) + 0.5), Y_k the real spherical harmonics with the
 *     Condon-Shortley phase, ordered l = 0..3, m = -l..l; dir = (mu - cam centre) / |.|.
 *   - alpha = min(0.99, opacity * exp(-0.5 d^T conic d)); a Gaussian contributes at a pixel
 *     iff alpha >= 1/255; blending stops before the first Gaussian that would take the
 *     transmittance below 1e-4 (that Gaussian is not blended).
 *   - depth = |mu_c| (distance along the ray); equal depths are ordered by Gaussian index.
 *   - footprint: q* = 2 ln(255 opacity); the ellipse d^T Sigma_p^-1 d <= q* has AABB
 *     half-extents sqrt(q* a), sqrt(q* c); padded by x(1 + 1e-5) + 1e-3 px; tile rect of
 *     16x16 tiles = floor((x -+ e) / 16), clamped to the grid, inclusive.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

#define ORC_NEAR 0.2
#define ORC_THETA_MAX (ORC_PI - 0.05)
#define ORC_THETA_MAX_ORTHO (0.5 * ORC_PI - 0.05)
#define ORC_PINHOLE_GUARD 1.3
#define ORC_LAT_MAX (0.5 * ORC_PI - 0.05)
#define ORC_CAM_EQUIDISTANT 0
#define ORC_CAM_EQUISOLID 1
#define ORC_CAM_STEREOGRAPHIC 2
#define ORC_CAM_ORTHOGRAPHIC 3
#define ORC_CAM_EQUIRECT 4
#define ORC_CAM_PINHOLE 5
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_ALPHA_MAX 0.99
#define ORC_T_MIN 1e-4
#define ORC_DILATION 0.3
#define ORC_TILE 16
#define ORC_SERIES_T 1e-2

/* Per-Gaussian record written by orc_project: ORC_NF doubles. */
#define ORC_NF 48
#define F_VIS 0
#define F_MUC 1   /* mu_c (3) */
#define F_XY 4    /* mu_p (2) */
#define F_J 6     /* J row-major 2x3 (6) */
#define F_SIG 12  /* Sigma: xx xy xz yy yz zz (6) */
#define F_COV 18  /* Sigma_p + 0.3 I: a b c (3) */
#define F_CON 21  /* conic A B C (3) */
#define F_OPA 24
#define F_RGB 25  /* clamped colour (3) */
#define F_RGBV 28 /* colour before the clamp (3) */
#define F_DEP 31
#define F_QST 32
#define F_EXT 33  /* padded AABB half-extents (2) */
#define F_RECT 35 /* tile rect x0 y0 x1 y1 (4), -1 when empty */
#define F_THETA 39
#define F_RMARG 40 /* distance (tiles) of the rect's floor() arguments to an integer */
#define F_DIR 41   /* view direction (3) */
#define F_CAMD 44  /* |mu - camera centre| */

int orc_nf(void) { return ORC_NF; }

/* camera: double[19] = W[9] (row-major, world -> camera), b[3], fx, fy, cx, cy, width, height,
 * model */

/* ---------------------------------------------------------------------------------------- */
/* Equidistant projection (Sec. 3.2) and its Jacobian (Sec. 4.2, f restored on theta terms). */

/* g = theta / l_z and h = (z l_z / l2 - theta) / l_z^3 = S7 / (l2^2 l_z^5), and
 * s8q = S8 / (l2^2 l_z^5). For 0 < t = l_z / z < 1e-2 the series
 *   theta / l_z          = z^-1 sum_{k>=0} (-1)^k t^{2k} / (2k+1)
 *   h                    = z^-3 sum_{k>=1} (-1)^k (2k / (2k+1)) t^{2k-2}
 *   S8 / (l2^2 l_z^5)    = (1/l_z) dh/dl_z = z^-5 sum_{k>=2} (-1)^k (2k/(2k+1)) (2k-2) t^{2k-4}
 * replace the cancelling closed forms; they follow from atan t = sum (-1)^k t^{2k+1}/(2k+1)
 * and t / (1 + t^2) = sum (-1)^k t^{2k+1}. */
static void orc_ghs(double x, double y, double z, double *theta, double *g, double *h,
                    double *s8q) {
  double lz2 = x * x + y * y, lz = sqrt(lz2), l2 = lz2 + z * z;
  double th = atan2(lz, z);
  *theta = th;
  if (z > 0 && lz < ORC_SERIES_T * z) {
    double t2 = lz2 / (z * z), z1 = 1.0 / z, z3 = z1 * z1 * z1, z5 = z3 * z1 * z1;
    double sg = 0, sh = 0, s8 = 0, p;
    int k;
    p = 1.0;
    for (k = 0; k < 10; ++k) { sg += ((k & 1) ? -1.0 : 1.0) * p / (2 * k + 1); p *= t2; }
    p = 1.0;
    for (k = 1; k < 10; ++k) { sh += ((k & 1) ? -1.0 : 1.0) * (2.0 * k / (2 * k + 1)) * p; p *= t2; }
    p = 1.0;
    for (k = 2; k < 11; ++k) {
      s8 += ((k & 1) ? -1.0 : 1.0) * (2.0 * k / (2 * k + 1)) * (2 * k - 2) * p; p *= t2;
    }
    *g = sg * z1; *h = sh * z3; *s8q = s8 * z5;
  } else {
    double lz3 = lz2 * lz, lz5 = lz3 * lz2, l22 = l2 * l2;
    double S7 = -l22 * lz2 * th + l2 * lz3 * z;
    double S8 = 3.0 * l22 * th - 3.0 * l2 * lz * z - 2.0 * lz3 * z;
    *g = th / lz;
    *h = S7 / (l22 * lz5);
    *s8q = S8 / (l22 * lz5);
  }
}

/* mu_p = phi(mu_c): x_p = c_x + f_x theta x_c / l_z, y_p = c_y + f_y theta y_c / l_z. */
void orc_project_point(const double *muc, double fx, double fy, double cx, double cy,
                       double *xy) {
  double th, g, h, s8;
  orc_ghs(muc[0], muc[1], muc[2], &th, &g, &h, &s8);
  xy[0] = cx + fx * g * muc[0];
  xy[1] = cy + fy * g * muc[1];
}

/* J_phi (2x3, row-major), the exact Jacobian of the projection above. */
void orc_jacobian(const double *muc, double fx, double fy, double *J) {
  double x = muc[0], y = muc[1], z = muc[2];
  double th, g, h, s8, l2 = x * x + y * y + z * z;
  orc_ghs(x, y, z, &th, &g, &h, &s8);
  J[0] = fx * (g + x * x * h); J[1] = fx * x * y * h; J[2] = -fx * x / l2;
  J[3] = fy * x * y * h; J[4] = fy * (g + y * y * h); J[5] = -fy * y / l2;
}

/* dJ/dx_c, dJ/dy_c, dJ/dz_c (each 2x3 row-major) in the paper's S1..S8 form, with
 * S7 / (l2^2 l_z^5) = h and S8 / (l2^2 l_z^5) = s8q, and dJ/dy_c[0,2] = 2 fx x y / l2^2. */
void orc_jacobian_grad(const double *muc, double fx, double fy, double *dJx, double *dJy,
                       double *dJz) {
  double x = muc[0], y = muc[1], z = muc[2];
  double th, g, h, s8q, l2 = x * x + y * y + z * z, l22 = l2 * l2;
  orc_ghs(x, y, z, &th, &g, &h, &s8q);
  /* S_i / (l2^2 l_z^5) for i = 1..4 */
  double s1 = x * (3.0 * h + x * x * s8q);
  double s2 = y * (h + x * x * s8q);
  double s3 = x * (h + y * y * s8q);
  double s4 = y * (3.0 * h + y * y * s8q);
  double S5 = x * x - y * y - z * z;
  double S6 = y * y - x * x - z * z;
  dJx[0] = fx * s1; dJx[1] = fx * s2; dJx[2] = fx * S5 / l22;
  dJx[3] = fy * s2; dJx[4] = fy * s3; dJx[5] = 2.0 * fy * x * y / l22;
  dJy[0] = fx * s2; dJy[1] = fx * s3; dJy[2] = 2.0 * fx * x * y / l22;
  dJy[3] = fy * s3; dJy[4] = fy * s4; dJy[5] = fy * S6 / l22;
  dJz[0] = fx * S5 / l22; dJz[1] = 2.0 * fx * x * y / l22; dJz[2] = 2.0 * fx * x * z / l22;
  dJz[3] = 2.0 * fy * x * y / l22; dJz[4] = fy * S6 / l22; dJz[5] = 2.0 * fy * y * z / l22;
}

/* ---------------------------------------------------------------------------------------- */
/* The other radial models: x_p = cx + fx g x, y_p = cy + fy g y with g = r(theta) / l_z, a
 * function G(l, z) of l = |mu_c| and z = z_c. With cos(theta) = z / l:
 *   equisolid      r = 2 sin(theta/2):  g = sqrt(2 / (l (l + z)))      (sin(theta/2)^2 = (l - z) / 2l)
 *   stereographic  r = 2 tan(theta/2):  g = 2 / (l + z)                (tan(theta/2) = l_z / (l + z))
 *   orthographic   r = sin(theta):      g = 1 / l                      (sin(theta) = l_z / l)
 *   pinhole        r = tan(theta):      g = 1 / z
 * G and its partial derivatives in (l, z) up to second order, from these closed forms. */
static void orc_radial_G(int model, double l, double z, double *G) {
  /* G[0..5] = G, G_l, G_z, G_ll, G_lz, G_zz */
  if (model == ORC_CAM_EQUISOLID) {
    double P = l * (l + z), Pl = 2 * l + z, Pz = l;  /* P_ll = 2, P_lz = 1, P_zz = 0 */
    double r2 = sqrt(2.0), Pm12 = 1.0 / sqrt(P), Pm32 = Pm12 / P, Pm52 = Pm32 / P;
    G[0] = r2 * Pm12;
    G[1] = -0.5 * r2 * Pm32 * Pl;
    G[2] = -0.5 * r2 * Pm32 * Pz;
    G[3] = 0.75 * r2 * Pm52 * Pl * Pl - 0.5 * r2 * Pm32 * 2.0;
    G[4] = 0.75 * r2 * Pm52 * Pl * Pz - 0.5 * r2 * Pm32 * 1.0;
    G[5] = 0.75 * r2 * Pm52 * Pz * Pz;
  } else if (model == ORC_CAM_STEREOGRAPHIC) {
    double S = l + z;
    G[0] = 2.0 / S;
    G[1] = G[2] = -2.0 / (S * S);
    G[3] = G[4] = G[5] = 4.0 / (S * S * S);
  } else if (model == ORC_CAM_PINHOLE) { /* x_p = cx + fx x / z: g = 1 / z */
    G[0] = 1.0 / z;
    G[1] = 0.0;
    G[2] = -1.0 / (z * z);
    G[3] = G[4] = 0.0;
    G[5] = 2.0 / (z * z * z);
  } else { /* orthographic */
    G[0] = 1.0 / l;
    G[1] = -1.0 / (l * l);
    G[2] = 0.0;
    G[3] = 2.0 / (l * l * l);
    G[4] = G[5] = 0.0;
  }
}

/* (g, h, k, h_l, h_z, k_l, k_z) of a radial model at mu_c, where g = G, h = G_l / l,
 * k = G_z + z h (so dg/dx = x h, dg/dz = k), h_l, k_l = (1/l) d/dl at fixed z, and h_z, k_z the
 * derivatives in z_c at fixed x_c, y_c. The equidistant model takes g, h, h_l from its series-
 * stabilised closed forms (h_l = S8 / (l2^2 l_z^5)), k = -1/l2, h_z = 2/l2^2, k_l = 2/l2^2,
 * k_z = 2 z / l2^2. */
static void orc_radial_terms(int model, double x, double y, double z, double *t) {
  double l2 = x * x + y * y + z * z, l = sqrt(l2);
  if (model == ORC_CAM_EQUIDISTANT) {
    double th, g, h, s8q;
    orc_ghs(x, y, z, &th, &g, &h, &s8q);
    t[0] = g; t[1] = h; t[2] = -1.0 / l2;
    t[3] = s8q; t[4] = 2.0 / (l2 * l2); t[5] = 2.0 / (l2 * l2); t[6] = 2.0 * z / (l2 * l2);
    return;
  }
  double G[6];
  orc_radial_G(model, l, z, G);
  double h = G[1] / l, k = G[2] + z * h;
  double Hl = G[3] / l - G[1] / (l * l), Hz = G[4] / l;
  double Kl = G[4] + z * Hl, Kz = G[5] + h + z * Hz;
  t[0] = G[0]; t[1] = h; t[2] = k;
  t[3] = Hl / l; t[4] = Hz + z * Hl / l; t[5] = Kl / l; t[6] = Kz + z * Kl / l;
}

/* Projection of mu_c for any model. */
void orc_cam_project(int model, const double *muc, double fx, double fy, double cx, double cy,
                     double *xy) {
  double x = muc[0], y = muc[1], z = muc[2];
  if (model == ORC_CAM_EQUIRECT) {
    xy[0] = cx + fx * atan2(x, z);
    xy[1] = cy + fy * atan2(y, sqrt(x * x + z * z));
    return;
  }
  double t[7];
  orc_radial_terms(model, x, y, z, t);
  xy[0] = cx + fx * t[0] * x;
  xy[1] = cy + fy * t[0] * y;
}

/* Jacobian (2x3 row-major) for any model. Panorama (Sec. 6, as printed there):
 *   [[fx z / rho^2, 0, -fx x / rho^2], [-fy x y / (rho l2), fy rho / l2, -fy y z / (rho l2)]],
 * rho = sqrt(x^2 + z^2). */
void orc_cam_jacobian(int model, const double *muc, double fx, double fy, double *J) {
  double x = muc[0], y = muc[1], z = muc[2];
  if (model == ORC_CAM_EQUIRECT) {
    double r2 = x * x + z * z, rho = sqrt(r2), l2 = r2 + y * y, u = 1.0 / (rho * l2);
    J[0] = fx * z / r2; J[1] = 0.0; J[2] = -fx * x / r2;
    J[3] = -fy * x * y * u; J[4] = fy * rho / l2; J[5] = -fy * y * z * u;
    return;
  }
  if (model == ORC_CAM_EQUIDISTANT) { orc_jacobian(muc, fx, fy, J); return; }
  double t[7];
  orc_radial_terms(model, x, y, z, t);
  double g = t[0], h = t[1], k = t[2];
  J[0] = fx * (g + x * x * h); J[1] = fx * x * y * h; J[2] = fx * x * k;
  J[3] = fy * x * y * h; J[4] = fy * (g + y * y * h); J[5] = fy * y * k;
}

/* dJ/dx_c, dJ/dy_c, dJ/dz_c for any model; the equidistant one in the paper's S1..S8 form
 * (orc_jacobian_grad), the other radial models from the terms of orc_radial_terms, the
 * panorama entry by entry. */
void orc_cam_jacobian_grad(int model, const double *muc, double fx, double fy, double *dJx,
                           double *dJy, double *dJz) {
  double x = muc[0], y = muc[1], z = muc[2];
  if (model == ORC_CAM_EQUIDISTANT) { orc_jacobian_grad(muc, fx, fy, dJx, dJy, dJz); return; }
  if (model == ORC_CAM_EQUIRECT) {
    double r2 = x * x + z * z, r4 = r2 * r2, rho = sqrt(r2), l2 = r2 + y * y;
    double u = 1.0 / (rho * l2), wq = 1.0 / r2 + 2.0 / l2;  /* du/dx = -x u wq, du/dz = -z u wq, du/dy = -2 y u / l2 */
    /* row 0: fx z / rho^2, 0, -fx x / rho^2 */
    dJx[0] = fx * (-2.0 * x * z / r4); dJy[0] = 0.0; dJz[0] = fx * (x * x - z * z) / r4;
    dJx[1] = 0.0; dJy[1] = 0.0; dJz[1] = 0.0;
    dJx[2] = fx * (x * x - z * z) / r4; dJy[2] = 0.0; dJz[2] = fx * 2.0 * x * z / r4;
    /* row 1: -fy x y u, fy rho / l2, -fy y z u */
    dJx[3] = fy * (-y * u + x * x * y * u * wq);
    dJy[3] = fy * (-x * u + 2.0 * x * y * y * u / l2);
    dJz[3] = fy * (x * y * z * u * wq);
    dJx[4] = fy * x * (u - 2.0 * rho / (l2 * l2));
    dJy[4] = fy * (-2.0 * y * rho / (l2 * l2));
    dJz[4] = fy * z * (u - 2.0 * rho / (l2 * l2));
    dJx[5] = fy * (x * y * z * u * wq);
    dJy[5] = fy * (-z * u + 2.0 * y * y * z * u / l2);
    dJz[5] = fy * (-y * u + y * z * z * u * wq);
    return;
  }
  double t[7];
  orc_radial_terms(model, x, y, z, t);
  double h = t[1], k = t[2], hl = t[3], hz = t[4], kl = t[5], kz = t[6];
  /* J00 = fx (g + x^2 h), J01 = fx x y h, J02 = fx x k; row 1 by x <-> y, fx -> fy */
  dJx[0] = fx * x * (3.0 * h + x * x * hl); dJy[0] = fx * y * (h + x * x * hl); dJz[0] = fx * (k + x * x * hz);
  dJx[1] = fx * y * (h + x * x * hl); dJy[1] = fx * x * (h + y * y * hl); dJz[1] = fx * x * y * hz;
  dJx[2] = fx * (k + x * x * kl); dJy[2] = fx * x * y * kl; dJz[2] = fx * x * kz;
  dJx[3] = fy * y * (h + x * x * hl); dJy[3] = fy * x * (h + y * y * hl); dJz[3] = fy * x * y * hz;
  dJx[4] = fy * x * (h + y * y * hl); dJy[4] = fy * y * (3.0 * h + y * y * hl); dJz[4] = fy * (k + y * y * hz);
  dJx[5] = fy * x * y * kl; dJy[5] = fy * (k + y * y * kl); dJz[5] = fy * y * kz;
}

/* Visibility angle test of a model: radial models bound theta, the panorama its latitude. */
static int orc_cam_in_field(int model, const double *muc, double *angle) {
  double x = muc[0], y = muc[1], z = muc[2];
  if (model == ORC_CAM_EQUIRECT) {
    double lat = atan2(fabs(y), sqrt(x * x + z * z));
    *angle = lat;
    return lat < ORC_LAT_MAX;
  }
  double th = atan2(sqrt(x * x + y * y), z);
  *angle = th;
  return th < ((model == ORC_CAM_ORTHOGRAPHIC || model == ORC_CAM_PINHOLE) ? ORC_THETA_MAX_ORTHO
                                                                          : ORC_THETA_MAX);
}

/* ---------------------------------------------------------------------------------------- */
/* Real spherical harmonics, degree <= 3, from their definition:
 *   Y_l^m = sqrt(2) K_l^|m| P_l^|m|(cos th) cos(m ph)   (m > 0)
 *         = sqrt(2) K_l^|m| P_l^|m|(cos th) sin(|m| ph) (m < 0)
 *         = K_l^0 P_l(cos th)                           (m = 0)
 * K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^m = (-1)^m sin^m(th) d^m P_l / dz^m.
 * sin^m(th) cos(m ph) + i sin^m(th) sin(m ph) = (d_x + i d_y)^m, so no angle is formed.
 * The polynomials of (d_x, d_y, d_z) are differentiated directly for the backward. */

static const double orc_legendre[4][4] = {
    /* coefficients of z^0..z^3 of P_0..P_3 (Bonnet: (l+1)P_{l+1} = (2l+1) z P_l - l P_{l-1}) */
    {1, 0, 0, 0}, {0, 1, 0, 0}, {-0.5, 0, 1.5, 0}, {0, -1.5, 0, 2.5}};

static double orc_fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }

/* value and derivative (in z) of d^m P_l / dz^m at z */
static void orc_legendre_dm(int l, int m, double z, double *v, double *dv) {
  double c[4] = {0, 0, 0, 0};
  for (int i = 0; i <= l; ++i) c[i] = orc_legendre[l][i];
  for (int r = 0; r < m; ++r) { for (int i = 0; i < 3; ++i) c[i] = (i + 1) * c[i + 1]; c[3] = 0; }
  *v = c[0] + z * (c[1] + z * (c[2] + z * c[3]));
  *dv = c[1] + z * (2 * c[2] + z * 3 * c[3]);
}

/* Y[k], k = l^2 + l + m, and dY/d(dir) [k][3] if dY != NULL. */
void orc_sh_basis(int degree, const double *d, double *Y, double *dY) {
  for (int l = 0; l <= degree; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m, k = l * l + l + m;
      double K = sqrt((2 * l + 1) / (4 * ORC_PI) * orc_fact(l - am) / orc_fact(l + am));
      double sgn = (am & 1) ? -1.0 : 1.0;
      double Pv, Pd;
      orc_legendre_dm(l, am, d[2], &Pv, &Pd);
      /* (d_x + i d_y)^am and its derivative am (d_x + i d_y)^(am-1) */
      double re = 1, im = 0, re1 = 0, im1 = 0;
      for (int r = 0; r < am; ++r) {
        if (r == am - 1) { re1 = am * re; im1 = am * im; }
        double nre = re * d[0] - im * d[1], nim = re * d[1] + im * d[0];
        re = nre; im = nim;
      }
      double c = (m == 0) ? K * sgn : sqrt(2.0) * K * sgn;
      double A, dAx, dAy;
      if (m > 0) { A = re; dAx = re1; dAy = -im1; }       /* d/dy of Re(w^m) = Re(i m w^{m-1}) */
      else if (m < 0) { A = im; dAx = im1; dAy = re1; }   /* d/dy of Im(w^m) = Im(i m w^{m-1}) */
      else { A = 1; dAx = 0; dAy = 0; }
      Y[k] = c * Pv * A;
      if (dY) {
        dY[3 * k + 0] = c * Pv * dAx;
        dY[3 * k + 1] = c * Pv * dAy;
        dY[3 * k + 2] = c * Pd * A;
      }
    }
  }
}

/* ---------------------------------------------------------------------------------------- */
/* Rotation from a quaternion (w, x, y, z), normalised first; row-major. */
static void orc_quat_to_R(const double *qn, double *R) {
  double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* 3x3 helpers (row-major) */
static void mm3(const double *A, const double *B, double *C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

static void orc_cam_centre(const double *cam, double *c) {
  /* c = -W^T b */
  for (int i = 0; i < 3; ++i) c[i] = -(cam[i] * cam[9] + cam[3 + i] * cam[10] + cam[6 + i] * cam[11]);
}

static double orc_tile_margin(double v) {
  double r = v - floor(v);
  return r < 1 - r ? r : 1 - r;
}

/* Per-Gaussian projection: out[n, ORC_NF]. Inputs are the values the method states:
 * means [n,3], scales [n,3] (activated, > 0), quats [n,4] (w,x,y,z, any norm),
 * opacities [n] (activated), sh [n, (degree+1)^2, 3]. */
void orc_project(int64_t n, const double *means, const double *scales, const double *quats,
                 const double *opac, const double *sh, int degree, const double *cam,
                 double *out) {
  const double *W = cam, *b = cam + 9;
  double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
  int width = (int)cam[16], height = (int)cam[17], model = (int)cam[18];
  int tiles_x = (width + ORC_TILE - 1) / ORC_TILE, tiles_y = (height + ORC_TILE - 1) / ORC_TILE;
  int nsh = (degree + 1) * (degree + 1);
  double cc[3];
  orc_cam_centre(cam, cc);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double *o = out + i * ORC_NF;
    memset(o, 0, sizeof(double) * ORC_NF);
    for (int k = 0; k < 4; ++k) o[F_RECT + k] = -1;
    const double *mu = means + 3 * i;
    double muc[3];
    for (int r = 0; r < 3; ++r) muc[r] = W[3 * r] * mu[0] + W[3 * r + 1] * mu[1] + W[3 * r + 2] * mu[2] + b[r];
    for (int r = 0; r < 3; ++r) o[F_MUC + r] = muc[r];
    double dist = sqrt(muc[0] * muc[0] + muc[1] * muc[1] + muc[2] * muc[2]);
    double angle;
    int in_field = orc_cam_in_field(model, muc, &angle);
    o[F_THETA] = angle;
    o[F_DEP] = dist;
    o[F_OPA] = opac[i];
    if (!(dist > ORC_NEAR) || !in_field || !(opac[i] >= ORC_ALPHA_MIN)) continue;

    orc_cam_project(model, muc, fx, fy, cx, cy, o + F_XY);
    /* the pinhole's guard band (distance to it kept as a decision margin, in tiles) */
    double guard_margin = 1e9;
    if (model == ORC_CAM_PINHOLE) {
      double gx = ORC_PINHOLE_GUARD * 0.5 * width - fabs(o[F_XY] - cx);
      double gy = ORC_PINHOLE_GUARD * 0.5 * height - fabs(o[F_XY + 1] - cy);
      if (!(gx >= 0 && gy >= 0)) continue;
      guard_margin = (gx < gy ? gx : gy) / ORC_TILE;
    }
    double J[6];
    orc_cam_jacobian(model, muc, fx, fy, J);
    memcpy(o + F_J, J, sizeof J);

    /* Sigma = R S S^T R^T */
    const double *q = quats + 4 * i;
    double qq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / qq, q[1] / qq, q[2] / qq, q[3] / qq}, R[9], M[9], Sig[9];
    orc_quat_to_R(qn, R);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * scales[3 * i + c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        Sig[3 * r + c] = M[3 * r] * M[3 * c] + M[3 * r + 1] * M[3 * c + 1] + M[3 * r + 2] * M[3 * c + 2];
    o[F_SIG + 0] = Sig[0]; o[F_SIG + 1] = Sig[1]; o[F_SIG + 2] = Sig[2];
    o[F_SIG + 3] = Sig[4]; o[F_SIG + 4] = Sig[5]; o[F_SIG + 5] = Sig[8];

    /* T = J W; Sigma_p = T Sigma T^T (+ 0.3 I) */
    double T[6], TS[6];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c)
        T[3 * r + c] = J[3 * r] * W[c] + J[3 * r + 1] * W[3 + c] + J[3 * r + 2] * W[6 + c];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c)
        TS[3 * r + c] = T[3 * r] * Sig[c] + T[3 * r + 1] * Sig[3 + c] + T[3 * r + 2] * Sig[6 + c];
    double a = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + ORC_DILATION;
    double bb = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    double c2 = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + ORC_DILATION;
    o[F_COV] = a; o[F_COV + 1] = bb; o[F_COV + 2] = c2;
    double det = a * c2 - bb * bb;
    o[F_CON] = c2 / det; o[F_CON + 1] = -bb / det; o[F_CON + 2] = a / det;

    /* colour from SH along dir = (mu - centre) / |mu - centre| */
    double dv[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double dir[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn}, Y[16];
    o[F_CAMD] = dn;
    for (int r = 0; r < 3; ++r) o[F_DIR + r] = dir[r];
    orc_sh_basis(degree, dir, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
      double v = 0.5;
      for (int k = 0; k < nsh; ++k) v += sh[(i * nsh + k) * 3 + ch] * Y[k];
      o[F_RGBV + ch] = v;
      o[F_RGB + ch] = v > 0 ? v : 0;
    }

    /* footprint: AABB of the alpha >= 1/255 ellipse, then the tile rect */
    double qs = 2.0 * log(255.0 * opac[i]);
    o[F_QST] = qs;
    double ex = sqrt(qs * a) * (1.0 + 1e-5) + 1e-3, ey = sqrt(qs * c2) * (1.0 + 1e-5) + 1e-3;
    o[F_EXT] = ex; o[F_EXT + 1] = ey;
    double x = o[F_XY], y = o[F_XY + 1];
    double lx = (x - ex) / ORC_TILE, hx = (x + ex) / ORC_TILE;
    double ly = (y - ey) / ORC_TILE, hy = (y + ey) / ORC_TILE;
    if (hx < 0 || hy < 0 || lx >= tiles_x || ly >= tiles_y) continue;
    double x0 = lx < 0 ? 0 : floor(lx), y0 = ly < 0 ? 0 : floor(ly);
    double x1 = floor(hx), y1 = floor(hy);
    if (x1 > tiles_x - 1) x1 = tiles_x - 1;
    if (y1 > tiles_y - 1) y1 = tiles_y - 1;
    double rm = guard_margin;
    if (lx >= 0) { double m = orc_tile_margin(lx); rm = m < rm ? m : rm; }
    if (ly >= 0) { double m = orc_tile_margin(ly); rm = m < rm ? m : rm; }
    if (hx < tiles_x) { double m = orc_tile_margin(hx); rm = m < rm ? m : rm; }
    if (hy < tiles_y) { double m = orc_tile_margin(hy); rm = m < rm ? m : rm; }
    o[F_RMARG] = rm;
    o[F_RECT] = x0; o[F_RECT + 1] = y0; o[F_RECT + 2] = x1; o[F_RECT + 3] = y1;
    o[F_VIS] = 1;
  }
}

/* ---------------------------------------------------------------------------------------- */
/* Per-pixel blending (Sec. 3.1 "Rendering"). */

typedef struct { double depth; int64_t idx; double alpha, araw, power; int contributes; } orc_cand;

static int orc_cand_cmp(const void *pa, const void *pb) {
  const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
  if (a->depth < b->depth) return -1;
  if (a->depth > b->depth) return 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Collect a pixel's candidates, sorted by (depth, index). A candidate is every visible
 * Gaussian with alpha >= 1/255 at the pixel ("contributes") plus those within the
 * decision band (|ln alpha_raw - ln(1/255)| < band) that only feed the margin.
 * use_bbox = 1 skips Gaussians whose padded AABB excludes the pixel centre; the AABB
 * contains the whole alpha >= 1/255 ellipse, so the contributing set is unchanged. */
static int64_t orc_collect(int64_t n, const double *G, double px, double py, int use_bbox,
                           double band, orc_cand **buf, int64_t *cap) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double *o = G + i * ORC_NF;
    if (o[F_VIS] == 0) continue;
    double dx = px - o[F_XY], dy = py - o[F_XY + 1];
    if (use_bbox && (fabs(dx) > o[F_EXT] || fabs(dy) > o[F_EXT + 1])) continue;
    double power = -0.5 * (o[F_CON] * dx * dx + 2.0 * o[F_CON + 1] * dx * dy + o[F_CON + 2] * dy * dy);
    double araw = o[F_OPA] * exp(power);
    double alpha = araw < ORC_ALPHA_MAX ? araw : ORC_ALPHA_MAX;
    int contributes = alpha >= ORC_ALPHA_MIN;
    if (!contributes && !(log(araw / ORC_ALPHA_MIN) > -band)) continue;
    if (m == *cap) { *cap = *cap ? 2 * *cap : 256; *buf = (orc_cand *)realloc(*buf, sizeof(orc_cand) * *cap); }
    orc_cand *c = *buf + m++;
    c->depth = o[F_DEP]; c->idx = i; c->alpha = alpha; c->araw = araw; c->power = power;
    c->contributes = contributes;
  }
  qsort(*buf, m, sizeof(orc_cand), orc_cand_cmp);
  return m;
}

/* Blend one pixel's sorted candidates. Returns the number blended; fills C, T_final, last
 * and the decision margins (relative distance of every alpha / T test that decided the
 * result from its threshold, and the relative depth gap of consecutive blended entries). */
/* Margins: each decision's relative distance from its threshold (log ratio for the alpha
 * and T tests, relative gap for the depth order), counted only when flipping that decision
 * could move the pixel's colour by at least impact_min: an alpha-threshold flip at
 * transmittance T changes the colour by about 2 T / 255 (its own term plus the dimming of
 * everything behind), a stop flip by about alpha T + 1e-4, a swap of two consecutive
 * Gaussians by about alpha_1 alpha_2 T. */
static int orc_blend(const double *G, const orc_cand *cand, int64_t m, const double *bg,
                     double impact_min, double *C, double *Tout, int64_t *last, double *m_alpha,
                     double *m_T, double *m_depth, double *Tbefore, int64_t *pos) {
  double T = 1.0, prev_depth = -1.0, prev_alpha = 0.0;
  int nb = 0;
  *m_alpha = *m_T = *m_depth = INFINITY;
  C[0] = C[1] = C[2] = 0;
  *last = -1;
  for (int64_t k = 0; k < m; ++k) {
    const orc_cand *c = cand + k;
    double ma = fabs(log(c->araw / ORC_ALPHA_MIN));
    if (ma < *m_alpha && 2.0 * T / 255.0 >= impact_min) *m_alpha = ma;
    if (!c->contributes) continue;
    double Tn = T * (1.0 - c->alpha);
    double mt = fabs(log(Tn / ORC_T_MIN));
    if (mt < *m_T && c->alpha * T + 1e-4 >= impact_min) *m_T = mt;
    if (prev_depth >= 0) {
      double md = (c->depth - prev_depth) / c->depth;
      if (md < *m_depth && prev_alpha * c->alpha * T >= impact_min) *m_depth = md;
    }
    prev_depth = c->depth;
    prev_alpha = c->alpha;
    if (Tn < ORC_T_MIN) break;
    const double *o = G + c->idx * ORC_NF;
    for (int ch = 0; ch < 3; ++ch) C[ch] += o[F_RGB + ch] * c->alpha * T;
    if (Tbefore) { Tbefore[nb] = T; pos[nb] = k; }
    T = Tn;
    *last = c->idx;
    ++nb;
  }
  for (int ch = 0; ch < 3; ++ch) C[ch] += T * bg[ch];
  *Tout = T;
  return nb;
}

/* Render pixels pix[npix][2] = (column i, row j), sampled at (i + 0.5, j + 0.5).
 * Outputs: color [npix,3], T_final [npix], last_g [npix] (index of the last blended
 * Gaussian, -1 if none), n_contrib [npix], margins [npix,3] (alpha, T, depth; log-ratio /
 * relative units; +inf when no decision of that kind, with impact >= impact_min, was taken). */
void orc_render(int64_t n, const double *G, int64_t npix, const int32_t *pix, const double *bg,
                int use_bbox, double band, double impact_min, double *color, double *T_final,
                int64_t *last_g, int32_t *n_contrib, double *margins) {
#pragma omp parallel
  {
    orc_cand *buf = NULL;
    int64_t cap = 0;
#pragma omp for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
      double px = pix[2 * p] + 0.5, py = pix[2 * p + 1] + 0.5;
      int64_t m = orc_collect(n, G, px, py, use_bbox, band, &buf, &cap);
      double ma, mt, md;
      n_contrib[p] = orc_blend(G, buf, m, bg, impact_min, color + 3 * p, T_final + p, last_g + p,
                               &ma, &mt, &md, NULL, NULL);
      margins[3 * p] = ma; margins[3 * p + 1] = mt; margins[3 * p + 2] = md;
    }
    free(buf);
  }
}

/* ---------------------------------------------------------------------------------------- */
/* Backward. L = sum_p <dLdC[p], C_p>.
 * Outputs (overwritten): d_means [n,3], d_scales [n,3], d_quats [n,4], d_opac [n],
 * d_sh [n,K,3]; and the screen-space intermediates g2d [n,9] =
 * (dL/dx_p, dL/dy_p, dL/dA, dL/dB, dL/dC of the conic, dL/dopacity, dL/drgb[3]). */
void orc_backward(int64_t n, const double *G, const double *means, const double *scales,
                  const double *quats, const double *opac, const double *sh, int degree,
                  const double *cam, int64_t npix, const int32_t *pix, const double *dLdC,
                  const double *bg, int use_bbox, double *d_means, double *d_scales,
                  double *d_quats, double *d_opac, double *d_sh, double *g2d) {
  int nsh = (degree + 1) * (degree + 1);
  memset(g2d, 0, sizeof(double) * 9 * n);
  (void)opac;
  (void)means;

  /* 1) per pixel, back to front through the blended list */
#pragma omp parallel
  {
    orc_cand *buf = NULL;
    int64_t cap = 0, tcap = 0, *pos = NULL;
    double *Tb = NULL;
#pragma omp for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
      const double *gC = dLdC + 3 * p;
      if (gC[0] == 0 && gC[1] == 0 && gC[2] == 0) continue;
      double px = pix[2 * p] + 0.5, py = pix[2 * p + 1] + 0.5;
      int64_t m = orc_collect(n, G, px, py, use_bbox, 0.0, &buf, &cap);
      if (m > tcap) {
        tcap = m;
        Tb = (double *)realloc(Tb, sizeof(double) * tcap);
        pos = (int64_t *)realloc(pos, sizeof(int64_t) * tcap);
      }
      double C[3], Tf, ma, mt, md;
      int64_t last;
      int nb = orc_blend(G, buf, m, bg, 0.0, C, &Tf, &last, &ma, &mt, &md, Tb, pos);
      /* S = colour behind blended entry k: sum_{j>k} rgb_j a_j T_j + T_final bg */
      double S[3] = {Tf * bg[0], Tf * bg[1], Tf * bg[2]};
      for (int k = nb - 1; k >= 0; --k) {
        const orc_cand *c = buf + pos[k];
        const double *o = G + c->idx * ORC_NF;
        double Tk = Tb[k], a = c->alpha;
        double dLda = 0;
        double *gg = g2d + 9 * c->idx;
        for (int ch = 0; ch < 3; ++ch) {
          double rgb = o[F_RGB + ch];
#pragma omp atomic
          gg[6 + ch] += gC[ch] * a * Tk;
          /* dC/dalpha_k = rgb_k T_k - S_k / (1 - alpha_k) */
          dLda += gC[ch] * (rgb * Tk - S[ch] / (1.0 - a));
          S[ch] += rgb * a * Tk;
        }
        if (c->araw < ORC_ALPHA_MAX) {
          /* alpha = opacity * exp(power), power = -0.5 (A dx^2 + 2 B dx dy + C dy^2) */
          double e_p = exp(c->power);
          double dLdp = dLda * a;
          double dx = px - o[F_XY], dy = py - o[F_XY + 1];
          double dxp = dLdp * (o[F_CON] * dx + o[F_CON + 1] * dy);
          double dyp = dLdp * (o[F_CON + 1] * dx + o[F_CON + 2] * dy);
          double dA = -0.5 * dx * dx * dLdp, dB = -dx * dy * dLdp, dCc = -0.5 * dy * dy * dLdp;
          double dop = dLda * e_p;
#pragma omp atomic
          gg[0] += dxp;
#pragma omp atomic
          gg[1] += dyp;
#pragma omp atomic
          gg[2] += dA;
#pragma omp atomic
          gg[3] += dB;
#pragma omp atomic
          gg[4] += dCc;
#pragma omp atomic
          gg[5] += dop;
        }
      }
    }
    free(buf);
    free(Tb);
    free(pos);
  }

  /* 2) per Gaussian, through the preprocess */
  const double *W = cam;
  double fx = cam[12], fy = cam[13];
  int model = (int)cam[18];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double *o = G + i * ORC_NF;
    double *dm = d_means + 3 * i, *ds = d_scales + 3 * i, *dq = d_quats + 4 * i;
    double *dsh = d_sh + (size_t)i * nsh * 3;
    memset(dm, 0, 3 * sizeof(double));
    memset(ds, 0, 3 * sizeof(double));
    memset(dq, 0, 4 * sizeof(double));
    memset(dsh, 0, sizeof(double) * nsh * 3);
    d_opac[i] = 0;
    if (o[F_VIS] == 0) continue;
    const double *gg = g2d + 9 * i;
    d_opac[i] = gg[5];

    /* colour -> SH coefficients and view direction */
    double Y[16], dY[48], ddir[3] = {0, 0, 0};
    orc_sh_basis(degree, o + F_DIR, Y, dY);
    for (int ch = 0; ch < 3; ++ch) {
      if (!(o[F_RGB + ch] > 0)) continue;
      double gr = gg[6 + ch];
      for (int k = 0; k < nsh; ++k) {
        dsh[3 * k + ch] = Y[k] * gr;
        double s = sh[(i * nsh + k) * 3 + ch] * gr;
        for (int r = 0; r < 3; ++r) ddir[r] += s * dY[3 * k + r];
      }
    }
    const double *dir = o + F_DIR;
    double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
    for (int r = 0; r < 3; ++r) dm[r] += (ddir[r] - dir[r] * dd) / o[F_CAMD];

    /* conic -> Sigma_p: dL/dSigma_p = -M Gc M (symmetric-matrix gradients), M = conic */
    double Mc[4] = {o[F_CON], o[F_CON + 1], o[F_CON + 1], o[F_CON + 2]};
    double Gc[4] = {gg[2], 0.5 * gg[3], 0.5 * gg[3], gg[4]};
    double t1[4], Gs[4];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) t1[2 * r + c] = Gc[2 * r] * Mc[c] + Gc[2 * r + 1] * Mc[2 + c];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) Gs[2 * r + c] = -(Mc[2 * r] * t1[c] + Mc[2 * r + 1] * t1[2 + c]);

    /* Sigma_p = T Sigma T^T: dL/dT = 2 Gs T Sigma, dL/dSigma = T^T Gs T */
    const double *J = o + F_J;
    double T[6], Sig[9];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c)
        T[3 * r + c] = J[3 * r] * W[c] + J[3 * r + 1] * W[3 + c] + J[3 * r + 2] * W[6 + c];
    Sig[0] = o[F_SIG]; Sig[1] = o[F_SIG + 1]; Sig[2] = o[F_SIG + 2];
    Sig[3] = o[F_SIG + 1]; Sig[4] = o[F_SIG + 3]; Sig[5] = o[F_SIG + 4];
    Sig[6] = o[F_SIG + 2]; Sig[7] = o[F_SIG + 4]; Sig[8] = o[F_SIG + 5];
    double GT[6], TS[6], GS3[9], GsT[6];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c)
        TS[3 * r + c] = T[3 * r] * Sig[c] + T[3 * r + 1] * Sig[3 + c] + T[3 * r + 2] * Sig[6 + c];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) GT[3 * r + c] = 2.0 * (Gs[2 * r] * TS[c] + Gs[2 * r + 1] * TS[3 + c]);
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) GsT[3 * r + c] = Gs[2 * r] * T[c] + Gs[2 * r + 1] * T[3 + c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) GS3[3 * r + c] = T[r] * GsT[c] + T[3 + r] * GsT[3 + c];

    /* T = J W: dL/dJ = dL/dT W^T */
    double GJ[6];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c)
        GJ[3 * r + c] = GT[3 * r] * W[3 * c] + GT[3 * r + 1] * W[3 * c + 1] + GT[3 * r + 2] * W[3 * c + 2];

    /* J -> mu_c through dJ/d{x,y,z}; mu_p -> mu_c through J^T (Sec. 4.2 and 4.3) */
    double dJx[6], dJy[6], dJz[6], dmuc[3] = {0, 0, 0};
    orc_cam_jacobian_grad(model, o + F_MUC, fx, fy, dJx, dJy, dJz);
    for (int e = 0; e < 6; ++e) {
      dmuc[0] += GJ[e] * dJx[e];
      dmuc[1] += GJ[e] * dJy[e];
      dmuc[2] += GJ[e] * dJz[e];
    }
    for (int r = 0; r < 3; ++r) dmuc[r] += J[r] * gg[0] + J[3 + r] * gg[1];
    /* mu_c = W mu + b: dL/dmu += W^T dL/dmu_c (summed with the colour path) */
    for (int c = 0; c < 3; ++c) dm[c] += W[c] * dmuc[0] + W[3 + c] * dmuc[1] + W[6 + c] * dmuc[2];

    /* Sigma = M M^T, M = R diag(s): dL/dM = 2 GS3 M */
    const double *q = quats + 4 * i;
    double qq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / qq, q[1] / qq, q[2] / qq, q[3] / qq}, R[9], M[9], GM[9];
    orc_quat_to_R(qn, R);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * scales[3 * i + c];
    mm3(GS3, M, GM);
    for (int e = 0; e < 9; ++e) GM[e] *= 2.0;
    double GR[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        ds[c] += GM[3 * r + c] * R[3 * r + c];
        GR[3 * r + c] = GM[3 * r + c] * scales[3 * i + c];
      }
    /* R(q) partial derivatives, entry by entry */
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    double gq[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; ++e) {
      gq[0] += GR[e] * dRw[e]; gq[1] += GR[e] * dRx[e];
      gq[2] += GR[e] * dRy[e]; gq[3] += GR[e] * dRz[e];
    }
    /* through q_n = q / |q| */
    double dot = gq[0] * qn[0] + gq[1] * qn[1] + gq[2] * qn[2] + gq[3] * qn[3];
    for (int r = 0; r < 4; ++r) dq[r] = (gq[r] - qn[r] * dot) / qq;
  }
}

/* ---------------------------------------------------------------------------------------- */
/* Tile binning and sort (the key definition): every record r with a non-empty rect emits,
 * for each tile (tx, ty) of its rect, key = ((tile_offset[view[r]] + ty * tiles_x[view[r]] + tx) << 32)
 * | depth_bits[r] and value r; the output is sorted by (key, value), i.e. the stable sort of
 * the emission in record order. tile_ranges[t] = [start, end) of global tile t.
 * Returns the number of pairs (capacity must be at least that; -1 otherwise). */
typedef struct { uint64_t key; uint32_t val; } orc_kv;

static int orc_kv_cmp(const void *pa, const void *pb) {
  const orc_kv *a = (const orc_kv *)pa, *b = (const orc_kv *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return (a->val > b->val) - (a->val < b->val);
}

/* Minimum over the rectangle [xl, xh] x [yl, yh] of q(d) = A dx^2 + 2 B dx dy + C dy^2,
 * d = p - mu, for a positive definite conic (A, B, C): 0 when mu lies in the rectangle, else
 * the smallest of the four edge minima (on an edge, the 1D minimiser of the free coordinate,
 * -B d_fixed / C or -B d_fixed / A, clamped to the edge). */
double orc_rect_min_q(const double *mu, const double *conic, double xl, double xh, double yl,
                      double yh) {
  double A = conic[0], B = conic[1], C = conic[2];
  if (mu[0] >= xl && mu[0] <= xh && mu[1] >= yl && mu[1] <= yh) return 0.0;
  double best = HUGE_VAL;
  for (int e = 0; e < 2; ++e) {
    double dx = (e ? xh : xl) - mu[0];
    double dy = -B * dx / C;
    if (dy < yl - mu[1]) dy = yl - mu[1];
    if (dy > yh - mu[1]) dy = yh - mu[1];
    double q = A * dx * dx + 2 * B * dx * dy + C * dy * dy;
    if (q < best) best = q;
    double ey = (e ? yh : yl) - mu[1];
    double ex = -B * ey / A;
    if (ex < xl - mu[0]) ex = xl - mu[0];
    if (ex > xh - mu[0]) ex = xh - mu[0];
    q = A * ex * ex + 2 * B * ex * ey + C * ey * ey;
    if (q < best) best = q;
  }
  return best;
}

/* Whether the exact binning keeps tile (tx, ty) of a record: the rectangle of the tile's pixel
 * centres against the level q* = 2 ln(255 opacity), with the margin q* (1 + 1e-3) + 1e-2. */
static int orc_keep_tile(const double *ell, int tx, int ty) {
  double xl = tx * ORC_TILE + 0.5, yl = ty * ORC_TILE + 0.5;
  double qs = ell[5] > 0 ? ell[5] : 0.0;
  return orc_rect_min_q(ell, ell + 2, xl, xl + ORC_TILE - 1, yl, yl + ORC_TILE - 1) <=
         qs * 1.001 + 1e-2;
}

/* ell: NULL (rect binning) or [nrec, 6] = mean x, y, conic A, B, C, q* (exact binning: only
 * the pairs orc_keep_tile accepts). */
int64_t orc_build_keys(int64_t nrec, const int32_t *view, const int32_t *rect /* [nrec,4] */,
                       const uint32_t *depth_bits, const int64_t *tile_offset,
                       const int32_t *tiles_x, int64_t n_tiles_total, int64_t capacity,
                       uint64_t *keys, uint32_t *vals, uint32_t *tile_ranges /* [n_tiles,2] */,
                       const double *ell) {
  int64_t m = 0;
  for (int64_t r = 0; r < nrec; ++r) {
    const int32_t *rc = rect + 4 * r;
    if (rc[0] < 0 || rc[2] < rc[0] || rc[3] < rc[1]) continue;
    for (int ty = rc[1]; ty <= rc[3]; ++ty)
      for (int tx = rc[0]; tx <= rc[2]; ++tx)
        if (!ell || orc_keep_tile(ell + 6 * r, tx, ty)) ++m;
  }
  if (m > capacity) return -1;
  orc_kv *kv = (orc_kv *)malloc(sizeof(orc_kv) * (m ? m : 1));
  int64_t e = 0;
  for (int64_t r = 0; r < nrec; ++r) {
    const int32_t *rc = rect + 4 * r;
    if (rc[0] < 0 || rc[2] < rc[0] || rc[3] < rc[1]) continue;
    for (int ty = rc[1]; ty <= rc[3]; ++ty)
      for (int tx = rc[0]; tx <= rc[2]; ++tx) {
        if (ell && !orc_keep_tile(ell + 6 * r, tx, ty)) continue;
        uint64_t tile = (uint64_t)(tile_offset[view[r]] + (int64_t)ty * tiles_x[view[r]] + tx);
        kv[e].key = (tile << 32) | depth_bits[r];
        kv[e].val = (uint32_t)r;
        ++e;
      }
  }
  qsort(kv, m, sizeof(orc_kv), orc_kv_cmp);
  for (int64_t t = 0; t < n_tiles_total; ++t) { tile_ranges[2 * t] = 0; tile_ranges[2 * t + 1] = 0; }
  for (int64_t k = 0; k < m; ++k) {
    keys[k] = kv[k].key;
    vals[k] = kv[k].val;
    int64_t t = (int64_t)(kv[k].key >> 32);
    if (k == 0 || (int64_t)(kv[k - 1].key >> 32) != t) tile_ranges[2 * t] = (uint32_t)k;
    tile_ranges[2 * t + 1] = (uint32_t)(k + 1);
  }
  free(kv);
  return m;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
