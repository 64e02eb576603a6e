/*
 * hot_oracle.c -- plain, slow, FP64 CPU oracle for weighted Gerchberg-Saxton (GSW)
 * hologram generation by direct superposition, after S. Bianchi and R. Di Leonardo,
 * "Real-time optical micro-manipulation using optimized holograms generated on the GPU".
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU
 * baseline may call this code. The product (the CUDA library) never links, loads or
 * falls back to it, and this file shares no code, header, table or constant with it.
 *
 * Every formula is evaluated literally, in double precision, with the C library's
 * sin/cos/atan2 (no fast math, no separability, no incremental phase, no caching of
 * Delta): a reader should be able to check each line against the paper.
 *
 * Conventions (readings where the paper is silent; the same readings are listed in
 * the design notes):
 *   - pixel j = iy*W + ix, coordinates x_j = (ix - floor(W/2)) * p,
 *     y_j = (iy - floor(H/2)) * p (the paper only says "coordinates of the j-th pixel",
 *     Sec. 3 after Eq. 2);
 *   - <|V|> in the weight update is the arithmetic mean of |V_m| over the trap index
 *     (Sec. 3, "averaging over the trap index m");
 *   - if |V_m| < 1e-30 the unit field V_m/|V_m| is taken as 1 and w_m is left unchanged;
 *   - arg(0) = atan2(0, 0) = 0, phases in (-pi, pi];
 *   - GSW order (flowchart of Fig. 2, whose image is lost): forward -> weight update
 *     (every iteration, the first included) -> back-projection; the reported V, e, u
 *     come from one more forward of the final phase.
 *
 * Parallelism: OpenMP over image rows. Every reduction over pixels is done as one
 * partial per row followed by a sum over rows in increasing row order, so the result
 * does not depend on the number of threads.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ---- threads ------------------------------------------------------------------ */

/* Sets the number of OpenMP threads when n > 0; returns the number in use. */
int oracle_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---- geometry ------------------------------------------------------------------ */

/* Pixel coordinate x_j (or y_j) of column ix (row iy) for an SLM of n columns (rows)
 * and pitch p; the origin is the pixel floor(n/2). */
static double pixel_coord(int i, int n, double p) { return (double)(i - n / 2) * p; }

/* Eq. 2: the phase acquired by light from pixel j to trap m,
 *   Delta_j^m = z_m pi / (lambda f^2) (x_j^2 + y_j^2) + 2 pi / (lambda f) (x_j x_m + y_j y_m). */
double oracle_delta(int W, int H, double p, double lam, double f, double xm, double ym,
                    double zm, int ix, int iy) {
  double xj = pixel_coord(ix, W, p), yj = pixel_coord(iy, H, p);
  return zm * ORACLE_PI / (lam * f * f) * (xj * xj + yj * yj) +
         2.0 * ORACLE_PI / (lam * f) * (xj * xm + yj * ym);
}

static int bad_geom(int W, int H, double p, double lam, double f) {
  return W <= 0 || H <= 0 || !(p > 0) || !(lam > 0) || !(f > 0);
}

/* ---- forward field (Eq. 1) ------------------------------------------------------ */

/* Eq. 1: V_m = (1/N) sum_j exp(i (phi_j - Delta_j^m)), for m = 0..M-1.
 * xyz: M*3 trap coordinates (x_m, y_m, z_m) in metres; phi: N pixel phases (rad);
 * V: 2*M output, interleaved (Re, Im). Returns 0, or -1 on invalid arguments. */
int oracle_forward(int W, int H, double p, double lam, double f, int M, const double *xyz,
                   const double *phi, double *V) {
  if (bad_geom(W, H, p, lam, f) || M < 1 || !xyz || !phi || !V) return -1;
  const long N = (long)W * H;
  double *rows = (double *)calloc((size_t)H * M * 2, sizeof(double));
  if (!rows) return -1;
#pragma omp parallel for schedule(static)
  for (int iy = 0; iy < H; iy++) {
    double *part = rows + (size_t)iy * M * 2;
    for (int m = 0; m < M; m++) {
      double re = 0.0, im = 0.0;
      for (int ix = 0; ix < W; ix++) {
        double d = oracle_delta(W, H, p, lam, f, xyz[3 * m], xyz[3 * m + 1], xyz[3 * m + 2], ix, iy);
        double a = phi[(long)iy * W + ix] - d;
        re += cos(a);
        im += sin(a);
      }
      part[2 * m] = re;
      part[2 * m + 1] = im;
    }
  }
  for (int m = 0; m < M; m++) {
    double re = 0.0, im = 0.0;
    for (int iy = 0; iy < H; iy++) {
      re += rows[((size_t)iy * M + m) * 2];
      im += rows[((size_t)iy * M + m) * 2 + 1];
    }
    V[2 * m] = re / (double)N;
    V[2 * m + 1] = im / (double)N;
  }
  free(rows);
  return 0;
}

/* ---- back-projection (Eq. 3 with complex trap coefficients) --------------------- */

/* Back-propagation from the traps to the SLM (Sec. 4, the step shared by SR and GSW):
 *   S_j = sum_m coef_m exp(i Delta_j^m),   phi_j = arg S_j.
 * SR (Eq. 3) is coef_m = exp(i theta_m); GSW uses coef_m = w_m V_m / |V_m|.
 * coef: 2*M interleaved; phi: N output phases in (-pi, pi] (may be NULL);
 * S: 2*N interleaved output superposition (may be NULL). */
int oracle_backproject(int W, int H, double p, double lam, double f, int M, const double *xyz,
                       const double *coef, double *phi, double *S) {
  if (bad_geom(W, H, p, lam, f) || M < 1 || !xyz || !coef || (!phi && !S)) return -1;
#pragma omp parallel for schedule(static)
  for (int iy = 0; iy < H; iy++) {
    for (int ix = 0; ix < W; ix++) {
      double re = 0.0, im = 0.0;
      for (int m = 0; m < M; m++) {
        double d = oracle_delta(W, H, p, lam, f, xyz[3 * m], xyz[3 * m + 1], xyz[3 * m + 2], ix, iy);
        double c = cos(d), s = sin(d);
        re += coef[2 * m] * c - coef[2 * m + 1] * s;
        im += coef[2 * m] * s + coef[2 * m + 1] * c;
      }
      long j = (long)iy * W + ix;
      if (phi) phi[j] = atan2(im, re);
      if (S) {
        S[2 * j] = re;
        S[2 * j + 1] = im;
      }
    }
  }
  return 0;
}

/* ---- weights (Sec. 3, GSW "update weights" box) ---------------------------------- */

/* w_m <- w_m <|V|> / |V_m| with <|V|> the mean of |V_m| over m, then
 * coef_m = w_m V_m / |V_m|. w is updated in place; coef (2*M) may be NULL.
 * If update == 0 only coef is formed from the current w. */
int oracle_update_weights(int M, const double *V, double *w, double *coef, int update) {
  if (M < 1 || !V || !w) return -1;
  double mean = 0.0;
  for (int m = 0; m < M; m++) mean += hypot(V[2 * m], V[2 * m + 1]);
  mean /= (double)M;
  for (int m = 0; m < M; m++) {
    double a = hypot(V[2 * m], V[2 * m + 1]);
    double ur = 1.0, ui = 0.0;
    if (a >= 1e-30) {
      ur = V[2 * m] / a;
      ui = V[2 * m + 1] / a;
      if (update) w[m] = w[m] * mean / a;
    }
    if (coef) {
      coef[2 * m] = w[m] * ur;
      coef[2 * m + 1] = w[m] * ui;
    }
  }
  return 0;
}

/* ---- efficiency and uniformity (Eq. 4) ------------------------------------------- */

/* I_m = |V_m|^2, e = sum_m I_m, u = 1 - (max I - min I) / (max I + min I).
 * If every I_m is zero, u is reported as 0. */
void oracle_metrics(int M, const double *V, double *e, double *u) {
  double s = 0.0, mx = -1.0, mn = 0.0;
  for (int m = 0; m < M; m++) {
    double I = V[2 * m] * V[2 * m] + V[2 * m + 1] * V[2 * m + 1];
    s += I;
    if (mx < 0.0 || I > mx) mx = I;
    if (m == 0 || I < mn) mn = I;
  }
  if (e) *e = s;
  if (u) *u = (mx + mn > 0.0) ? 1.0 - (mx - mn) / (mx + mn) : 0.0;
}

/* ---- the GSW iteration (Sec. 3, Fig. 2) ------------------------------------------ */

/* K iterations of GSW starting from phases phi (N, in/out) and weights w (M, in/out):
 *   for k = 1..K:  V = F(phi);  w <- w <|V|>/|V|;  phi = arg sum_m w_m V_m/|V_m| e^{i Delta}.
 * Afterwards V (2*M, may be NULL) = F(phi^K) and e, u (may be NULL) from Eq. 4.
 * Calling it twice with K1 and K2 gives the same state as one call with K1 + K2. */
int oracle_gsw(int W, int H, double p, double lam, double f, int M, const double *xyz, int K,
               double *phi, double *w, double *V, double *e, double *u) {
  if (bad_geom(W, H, p, lam, f) || M < 1 || K < 0 || !xyz || !phi || !w) return -1;
  double *Vk = (double *)malloc(sizeof(double) * 2 * M);
  double *coef = (double *)malloc(sizeof(double) * 2 * M);
  if (!Vk || !coef) {
    free(Vk);
    free(coef);
    return -1;
  }
  int rc = 0;
  for (int k = 0; k < K && rc == 0; k++) {
    rc = oracle_forward(W, H, p, lam, f, M, xyz, phi, Vk);
    if (rc == 0) rc = oracle_update_weights(M, Vk, w, coef, 1);
    if (rc == 0) rc = oracle_backproject(W, H, p, lam, f, M, xyz, coef, phi, NULL);
  }
  if (rc == 0 && (V || e || u)) {
    rc = oracle_forward(W, H, p, lam, f, M, xyz, phi, Vk);
    if (rc == 0) {
      if (V) memcpy(V, Vk, sizeof(double) * 2 * M);
      oracle_metrics(M, Vk, e, u);
    }
  }
  free(Vk);
  free(coef);
  return rc;
}

/* ---- 8-bit SLM encoding (Sec. 5) -------------------------------------------------- */

/* Grey levels are mapped linearly onto phase 0..2pi. Reading: 256 levels of width
 * 2pi/256, level 0 == phase 0 == 2pi, round to nearest (ties to even):
 *   g_j = rint(phi_j * 256 / (2 pi)) mod 256, taken non-negative. */
void oracle_quantize(long N, const double *phi, unsigned char *g) {
  for (long j = 0; j < N; j++) {
    double q = rint(phi[j] * 256.0 / (2.0 * ORACLE_PI));
    long k = ((long)q) % 256;
    if (k < 0) k += 256;
    g[j] = (unsigned char)k;
  }
}

/* ---- adjoint of Eq. 1 (gradient of a real loss of V with respect to phi) ----------- */

/* For a real loss L(V) with G_m = 2 dL/d(conj V_m) (2*M interleaved), the gradient is
 *   dL/dphi_j = (1/N) Im[ exp(-i phi_j) sum_m G_m exp(i Delta_j^m) ],
 * obtained by differentiating Eq. 1: dV_m/dphi_j = (i/N) exp(i(phi_j - Delta_j^m)). */
int oracle_adjoint(int W, int H, double p, double lam, double f, int M, const double *xyz,
                   const double *phi, const double *G, double *grad) {
  if (bad_geom(W, H, p, lam, f) || M < 1 || !xyz || !phi || !G || !grad) return -1;
  const long N = (long)W * H;
#pragma omp parallel for schedule(static)
  for (int iy = 0; iy < H; iy++) {
    for (int ix = 0; ix < W; ix++) {
      double re = 0.0, im = 0.0;
      for (int m = 0; m < M; m++) {
        double d = oracle_delta(W, H, p, lam, f, xyz[3 * m], xyz[3 * m + 1], xyz[3 * m + 2], ix, iy);
        double c = cos(d), s = sin(d);
        re += G[2 * m] * c - G[2 * m + 1] * s;
        im += G[2 * m] * s + G[2 * m + 1] * c;
      }
      long j = (long)iy * W + ix;
      /* Im[(cos phi - i sin phi)(re + i im)] = cos(phi) im - sin(phi) re */
      grad[j] = (cos(phi[j]) * im - sin(phi[j]) * re) / (double)N;
    }
  }
  return 0;
}
