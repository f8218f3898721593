/*
 * CPU oracle for the per-job arithmetic of the SET executor's workloads.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this file.  It
 * shares no code, header, table or constant with the CUDA path; both read the
 * same seeded inputs from the datagen module and nothing else.
 *
 * Every function is the plain definition of its stage, run serially, one pixel
 * or element at a time, in the order the definition states.  Floating-point
 * accumulations that the GPU reassociates are carried in fp64 here.
 *
 * The SET paper (Li, Huang, Ogras) treats each job as an opaque chain
 * H2D -> stage kernels -> D2H (Sec. 3.2, Eq. 1) and names image-filter, scan-like
 * and GEMM workloads (Sec. 5.1.2); it prints no stage arithmetic.  The stages
 * below are the executor's synthetic workloads:
 *   blur job : 3x3 box blur (integer sum / 9, floored, edge-clamped) -> 256-bin histogram
 *   scan job : z = fmaf(a, x, y) -> exclusive prefix sum S -> m = max |S_i|
 *   img job  : gray = (77R + 150G + 29B) >> 8 -> 5x5 Gaussian [1,4,6,4,1] (x) [1,4,6,4,1] >> 8
 *              -> Sobel min(|gx| + |gy|, 255) -> 256-bin histogram
 *   hotspot  : K explicit Euler steps of a compact thermal RC grid (fp64 here)
 * (The MLP job's oracle is oracle/mlp.py, fp64 numpy.)
 * Every stencil clamps its own input image at the border (replicate edge).
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off (no FMA contraction, so that
 * fp64 sums are the same on x86-64 and aarch64).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

/* 3x3 box blur: o[y][x] = floor( sum_{dy,dx in -1..1} I[cl(y+dy)][cl(x+dx)] / 9 ). */
void oracle_blur3x3(const uint8_t* in, int W, int H, uint8_t* out) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      unsigned s = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) s += in[(size_t)clampi(y + dy, H) * W + clampi(x + dx, W)];
      out[(size_t)y * W + x] = (uint8_t)(s / 9u);
    }
}

/* 256-bin histogram: h[v] = #{p : img[p] == v}. */
void oracle_hist256(const uint8_t* img, size_t n, uint32_t* hist) {
  memset(hist, 0, 256 * sizeof(uint32_t));
  for (size_t p = 0; p < n; ++p) hist[img[p]] += 1;
}

/* saxpy: z_i = fmaf(a, x_i, y_i), the correctly rounded fp32 fused multiply-add. */
void oracle_saxpy(float a, const float* x, const float* y, size_t n, float* z) {
  for (size_t i = 0; i < n; ++i) z[i] = fmaf(a, x[i], y[i]);
}

/* Exclusive prefix sum in fp64: S_0 = 0, S_i = sum_{j<i} z_j.  Also returns the
 * running absolute sum A_i = sum_{j<i} |z_j| that bounds any reassociated fp32
 * evaluation (|S_gpu - S| <= c * eps32 * A_i). */
void oracle_exscan(const float* z, size_t n, double* S, double* A) {
  double s = 0.0, a = 0.0;
  for (size_t i = 0; i < n; ++i) {
    S[i] = s;
    if (A) A[i] = a;
    s += (double)z[i];
    a += fabs((double)z[i]);
  }
}

/* m = max_i |S_i| over the scan output. */
double oracle_maxabs(const double* S, size_t n) {
  double m = 0.0;
  for (size_t i = 0; i < n; ++i) m = fmax(m, fabs(S[i]));
  return m;
}

/* Gray: g = (77 R + 150 G + 29 B) >> 8 on interleaved RGB (row-major, no padding). */
void oracle_gray(const uint8_t* rgb, int W, int H, uint8_t* g) {
  for (size_t p = 0; p < (size_t)W * H; ++p) {
    const unsigned r = rgb[3 * p], gg = rgb[3 * p + 1], b = rgb[3 * p + 2];
    g[p] = (uint8_t)((77u * r + 150u * gg + 29u * b) >> 8);
  }
}

/* 5x5 Gaussian: q[y][x] = ( sum_{i,j in -2..2} w_i w_j g[cl(y+i)][cl(x+j)] ) >> 8,
 * w = [1, 4, 6, 4, 1]; one shift of the full 2-D sum (weights sum to 256). */
void oracle_gauss5(const uint8_t* g, int W, int H, uint8_t* q) {
  static const unsigned w[5] = {1, 4, 6, 4, 1};
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      unsigned s = 0;
      for (int i = -2; i <= 2; ++i)
        for (int j = -2; j <= 2; ++j)
          s += w[i + 2] * w[j + 2] * g[(size_t)clampi(y + i, H) * W + clampi(x + j, W)];
      q[(size_t)y * W + x] = (uint8_t)(s >> 8);
    }
}

/* Sobel: gx with kernel [[-1,0,1],[-2,0,2],[-1,0,1]], gy its transpose
 * (top row negative), s = min(|gx| + |gy|, 255), clamped borders. */
void oracle_sobel(const uint8_t* q, int W, int H, uint8_t* s) {
  static const int kx[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
  static const int ky[3][3] = {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}};
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int gx = 0, gy = 0;
      for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j) {
          const int v = q[(size_t)clampi(y + i, H) * W + clampi(x + j, W)];
          gx += kx[i + 1][j + 1] * v;
          gy += ky[i + 1][j + 1] * v;
        }
      const int m = abs(gx) + abs(gy);
      s[(size_t)y * W + x] = (uint8_t)(m > 255 ? 255 : m);
    }
}

/* ---- whole jobs: the stages of one job run serially, in chain order ---- */

/* blur job: blurred (W*H bytes) and its histogram (256 u32). */
void oracle_job_blur_hist(const uint8_t* img, int W, int H, uint8_t* blurred, uint32_t* hist) {
  oracle_blur3x3(img, W, H, blurred);
  oracle_hist256(blurred, (size_t)W * H, hist);
}

/* scan job: z (fp32, exact), S (fp64), A (fp64 bound, may be NULL), returns m. */
double oracle_job_saxpy_scan_max(float a, const float* x, const float* y, size_t n, float* z,
                                 double* S, double* A) {
  oracle_saxpy(a, x, y, n, z);
  oracle_exscan(z, n, S, A);
  return oracle_maxabs(S, n);
}

/* img job: Sobel image (W*H bytes) and its histogram; gray and gauss are
 * caller-provided W*H work buffers. */
void oracle_job_img_sobel_hist(const uint8_t* rgb, int W, int H, uint8_t* gray, uint8_t* gauss,
                               uint8_t* sobel, uint32_t* hist) {
  oracle_gray(rgb, W, H, gray);
  oracle_gauss5(gray, W, H, gauss);
  oracle_sobel(gauss, W, H, sobel);
  oracle_hist256(sobel, (size_t)W * H, hist);
}

/* ---- hotspot job ----
 *
 * Sec. 5.1.2 names Hotspot (the HotSpot compact thermal model of Huang et al.,
 * 2006): iterative thermal simulation.  The paper gives no parameters; the job
 * is the model's R x C grid of cells over a silicon die, advanced K explicit
 * Euler steps.  With dx = die width / C and dy = die height / R:
 *   Gx  = k t dy / dx   conductance to each left / right neighbour
 *   Gy  = k t dx / dy   conductance to each upper / lower neighbour
 *   Gz  = k dx dy / t   conductance to the ambient through the die's thickness
 *   Cap = c_v t dx dy   heat capacity of a cell
 *   dt  = 0.2 Cap / (2 Gx + 2 Gy + Gz)   (a fifth of the scheme's positivity limit)
 *   T'  = T + dt / Cap * (P + Gy (T_N + T_S - 2 T) + Gx (T_W + T_E - 2 T) + Gz (T_amb - T))
 * A neighbour outside the die is the cell itself (adiabatic edges: no flux).
 * Die 16 mm x 16 mm x 0.5 mm, k = 100 W/(m K), c_v = 1.75e6 J/(m^3 K),
 * T_amb = 80.  T in degrees, P in watts per cell.  Evaluated in fp64 from the
 * fp32 inputs, in the order written above. */
#define ORACLE_HOT_DIE_W 0.016
#define ORACLE_HOT_DIE_H 0.016
#define ORACLE_HOT_THICK 0.0005
#define ORACLE_HOT_K_SI 100.0
#define ORACLE_HOT_CV_SI 1.75e6
#define ORACLE_HOT_T_AMB 80.0
#define ORACLE_HOT_DT_FRAC 0.2

/* c = {Gx, Gy, Gz, Cap, dt, T_amb} of an R x C grid. */
void oracle_hotspot_params(int R, int C, double* c) {
  const double dx = ORACLE_HOT_DIE_W / C, dy = ORACLE_HOT_DIE_H / R;
  const double gx = ORACLE_HOT_K_SI * ORACLE_HOT_THICK * dy / dx;
  const double gy = ORACLE_HOT_K_SI * ORACLE_HOT_THICK * dx / dy;
  const double gz = ORACLE_HOT_K_SI * dx * dy / ORACLE_HOT_THICK;
  const double cap = ORACLE_HOT_CV_SI * ORACLE_HOT_THICK * dx * dy;
  c[0] = gx;
  c[1] = gy;
  c[2] = gz;
  c[3] = cap;
  c[4] = ORACLE_HOT_DT_FRAC * cap / (2.0 * gx + 2.0 * gy + gz);
  c[5] = ORACLE_HOT_T_AMB;
}

/* T (R*C doubles, row-major) = the grid after K steps from T0 under power P. */
void oracle_hotspot(const float* T0, const float* P, int R, int C, int K, double* T) {
  double c[6];
  oracle_hotspot_params(R, C, c);
  const double gx = c[0], gy = c[1], gz = c[2], cap = c[3], dt = c[4], tamb = c[5];
  const size_t n = (size_t)R * C;
  double* cur = (double*)malloc(n * sizeof(double));
  double* nxt = (double*)malloc(n * sizeof(double));
  for (size_t i = 0; i < n; ++i) cur[i] = (double)T0[i];
  for (int step = 0; step < K; ++step) {
    for (int i = 0; i < R; ++i)
      for (int j = 0; j < C; ++j) {
        const double t = cur[(size_t)i * C + j];
        const double tn = cur[(size_t)clampi(i - 1, R) * C + j], ts = cur[(size_t)clampi(i + 1, R) * C + j];
        const double tw = cur[(size_t)i * C + clampi(j - 1, C)], te = cur[(size_t)i * C + clampi(j + 1, C)];
        const double p = (double)P[(size_t)i * C + j];
        nxt[(size_t)i * C + j] =
            t + dt / cap * (p + gy * (tn + ts - 2.0 * t) + gx * (tw + te - 2.0 * t) + gz * (tamb - t));
      }
    double* sw = cur;
    cur = nxt;
    nxt = sw;
  }
  memcpy(T, cur, n * sizeof(double));
  free(cur);
  free(nxt);
}
