/* synth.c — seeded synthetic images shaped like the paper's workloads.
 *
 * Holds no codec arithmetic: it only draws pixels.  Both the CPU oracle
 * (tests, CPU baseline) and the GPU library consume the bytes it writes.
 *
 * Every image is a pure function of (seed, pixel position): a counter-based
 * splitmix64 hash gives each lattice point, cell and pixel its own random
 * numbers, so any crop can be generated on its own and in parallel.
 * Only +, -, *, /, sqrt, rint, floor and fabs are used on doubles, and bit
 * reads of the exponent (correctly rounded or exact under IEEE 754) and the file is compiled
 * with -ffp-contract=off, so the bytes are identical on x86-64 and AArch64
 * hosts.
 *
 *   isx_gen_stain    512x512-style RGB8 tile: near-white base, smooth colour
 *                    gradients, pink/purple stain hues, N(0, 8^2) noise.
 *   isx_gen_slide    whole-slide-shaped RGB8: ~60% pale background
 *                    (230..250, N(0, 3^2)), tissue of pink stroma with dark
 *                    purple nuclei discs of radius 3..8 px, N(0, 10^2).
 *   isx_gen_phantom  12-bit monochrome in uint16: smooth elliptical phantoms
 *                    (values 0..4095, summed then clamped) whose value v at
 *                    a pixel is replaced by a Poisson(v) sample.
 * Gaussian deviates come from the Box-Muller transform (one deviate per
 * pixel and channel: sqrt(-2 ln u1) cos(2 pi u2)), Poisson samples from
 * exponential inter-arrival counting for small means and from Hormann's
 * transformed rejection with squeeze (1993) for means of 10 and above.  The
 * logarithm, cosine and log-factorial they need are written out below as
 * polynomials in +, -, * and / only (after an exact split of the exponent),
 * so that they keep the bytes identical across hosts as well.
 */
#include <stdint.h>
#include <math.h>
#include <pthread.h>
#include <string.h>

static inline uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
static inline uint64_t key3(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
  return mix64(mix64(mix64(seed ^ 0x243F6A8885A308D3ull) ^ a) ^ (b * 0x9E3779B97F4A7C15ull) ^ (c << 17));
}
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

static const double kLn2 = 0.69314718055994530942, kHalfPi = 1.57079632679489661923;

/* natural logarithm of x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + ... + s^20/21) with
 * s = (m-1)/(m+1), |s| <= 0.1716 (the next term is below 2^-56); Horner
 * form, the coefficients 1/(2j+1) folded by the compiler (correctly
 * rounded, so the same on every host) */
static double ln_d(double x) {
  /* x = m 2^e, m in [1/2, 1), read from the bits (exact) */
  uint64_t bits;
  memcpy(&bits, &x, 8);
  int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0) {   /* subnormal: scale by 2^54 first */
    x *= 18014398509481984.0;
    memcpy(&bits, &x, 8);
    e = (int)((bits >> 52) & 0x7ff) - 54;
  }
  e -= 1022;
  bits = (bits & 0x800FFFFFFFFFFFFFull) | 0x3FE0000000000000ull;
  double m;
  memcpy(&m, &bits, 8);
  if (m < 0.70710678118654752440) {
    m *= 2.0;
    e -= 1;
  }
  const double s = (m - 1.0) / (m + 1.0), s2 = s * s;
  double p = 1.0 / 21.0;
  p = p * s2 + 1.0 / 19.0;
  p = p * s2 + 1.0 / 17.0;
  p = p * s2 + 1.0 / 15.0;
  p = p * s2 + 1.0 / 13.0;
  p = p * s2 + 1.0 / 11.0;
  p = p * s2 + 1.0 / 9.0;
  p = p * s2 + 1.0 / 7.0;
  p = p * s2 + 1.0 / 5.0;
  p = p * s2 + 1.0 / 3.0;
  p = p * s2 + 1.0;
  return 2.0 * s * p + (double)e * kLn2;
}

/* cos(2 pi u) for u in [0, 1): u in quarter turns t = 4u = q + r with q
 * the nearest integer, |r| <= 1/2, angle a = r pi/2 (|a| <= pi/4), cos a
 * and sin a by their Taylor polynomials to a^16 and a^17 (Horner, the
 * coefficients 1/n! folded by the compiler), the quadrant by symmetry */
static double cos_2pi(double u) {
  const double t = 4.0 * u, q = rint(t);
  const double a = (t - q) * kHalfPi, a2 = a * a;
  double c = 1.0 / 20922789888000.0;              /* 1/16! */
  c = c * a2 - 1.0 / 87178291200.0;               /* 1/14! */
  c = c * a2 + 1.0 / 479001600.0;                 /* 1/12! */
  c = c * a2 - 1.0 / 3628800.0;
  c = c * a2 + 1.0 / 40320.0;
  c = c * a2 - 1.0 / 720.0;
  c = c * a2 + 1.0 / 24.0;
  c = c * a2 - 1.0 / 2.0;
  c = c * a2 + 1.0;
  double sn = 1.0 / 355687428096000.0;            /* 1/17! */
  sn = sn * a2 - 1.0 / 1307674368000.0;           /* 1/15! */
  sn = sn * a2 + 1.0 / 6227020800.0;              /* 1/13! */
  sn = sn * a2 - 1.0 / 39916800.0;
  sn = sn * a2 + 1.0 / 362880.0;
  sn = sn * a2 - 1.0 / 5040.0;
  sn = sn * a2 + 1.0 / 120.0;
  sn = sn * a2 - 1.0 / 6.0;
  sn = sn * a2 + 1.0;
  sn *= a;
  switch (((int)q) & 3) {
    case 0: return c;
    case 1: return -sn;
    case 2: return -c;
    default: return sn;
  }
}

/* standard normal deviate, Box-Muller: u1 in (0, 1], u2 in [0, 1) */
static inline double gauss(uint64_t key) {
  const uint64_t a = mix64(key), b = mix64(key ^ 0xD1B54A32D192ED03ull);
  const double u1 = (double)((a >> 11) + 1) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * ln_d(u1)) * cos_2pi(u2);
}

/* ln k! : the sum of logarithms below 10, Stirling's series above
 * (ln Gamma(x) = (x - 1/2) ln x - x + ln(2 pi)/2 + 1/(12x) - 1/(360x^3)
 * + 1/(1260x^5) - 1/(1680x^7), x = k + 1 >= 11) */
static double ln_fact(int64_t k) {
  if (k < 10) {
    double s = 0.0;
    for (int64_t i = 2; i <= k; ++i) s += ln_d((double)i);
    return s;
  }
  const double x = (double)(k + 1), x2 = x * x;
  return (x - 0.5) * ln_d(x) - x + 0.91893853320467274178 +
         (1.0 / 12.0 - (1.0 / 360.0 - (1.0 / 1260.0 - (1.0 / 1680.0) / x2) / x2) / x2) / x;
}

/* the i-th uniform of the stream `key`, in (0, 1] */
static inline double u01_open0(uint64_t key, uint64_t i) {
  return (double)((mix64(key + i * 0x9E3779B97F4A7C15ull) >> 11) + 1) * (1.0 / 9007199254740992.0);
}

/* Poisson(lam) sample from the uniform stream `key` */
static int64_t poisson(double lam, uint64_t key) {
  if (lam <= 0.0) return 0;
  if (lam < 10.0) {
    /* arrivals of a unit-rate Poisson process before time lam: the
     * inter-arrival times are -ln u */
    double tsum = 0.0;
    int64_t k = 0;
    for (uint64_t i = 0; i < 1000; ++i) {
      tsum -= ln_d(u01_open0(key, i));
      if (tsum > lam) break;
      ++k;
    }
    return k;
  }
  /* transformed rejection with squeeze (Hormann 1993) */
  const double slam = sqrt(lam), loglam = ln_d(lam);
  const double b = 0.931 + 2.53 * slam, a = -0.059 + 0.02483 * b;
  const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4), vr = 0.9277 - 3.6224 / (b - 2.0);
  int64_t k = (int64_t)floor(lam);   /* returned only if every try is rejected (the bound only guards the loop) */
  for (uint64_t i = 0; i < 256; i += 2) {
    const double U = u01_open0(key, i) - 0.5, V = u01_open0(key, i + 1);
    const double us = 0.5 - fabs(U);
    if (us <= 0.0) continue;   /* U = 1/2 (probability 2^-53): no k */
    const double kd = floor((2.0 * a / us + b) * U + lam + 0.43);
    if (us >= 0.07 && V <= vr) return (int64_t)kd;
    if (kd < 0.0 || kd > 1e9 || (us < 0.013 && V > us)) continue;
    k = (int64_t)kd;
    if (ln_d(V) + ln_d(inv_alpha) - ln_d(a / (us * us) + b) <= -lam + (double)k * loglam - ln_fact(k)) return k;
  }
  return k < 0 ? 0 : k;
}

/* smooth value noise in [0,1): random values on a lattice of spacing sp,
 * blended with the smoothstep weights 3t^2 - 2t^3 */
static double vnoise(uint64_t seed, int64_t x, int64_t y, int64_t sp) {
  int64_t gx = x / sp, gy = y / sp;
  double tx = (double)(x - gx * sp) / (double)sp, ty = (double)(y - gy * sp) / (double)sp;
  double sx = tx * tx * (3.0 - 2.0 * tx), sy = ty * ty * (3.0 - 2.0 * ty);
  double v00 = u01(key3(seed, 11, (uint64_t)gx, (uint64_t)gy));
  double v10 = u01(key3(seed, 11, (uint64_t)gx + 1, (uint64_t)gy));
  double v01 = u01(key3(seed, 11, (uint64_t)gx, (uint64_t)gy + 1));
  double v11 = u01(key3(seed, 11, (uint64_t)gx + 1, (uint64_t)gy + 1));
  double a = v00 + (v10 - v00) * sx, b = v01 + (v11 - v01) * sx;
  return a + (b - a) * sy;
}

static inline int clampi(double v, int lo, int hi) {
  double r = rint(v);
  if (r < lo) return lo;
  if (r > hi) return hi;
  return (int)r;
}

/* ---------------------------------------------------------------- stain */
static void stain_row(uint64_t seed, int64_t y, int64_t w, uint8_t* row) {
  /* 2..4 linear colour gradients, fixed per seed */
  int ng = 2 + (int)(mix64(seed ^ 0x51) % 3);
  for (int64_t x = 0; x < w; ++x) {
    double col[3] = {240.0, 240.0, 240.0};
    for (int g = 0; g < ng; ++g) {
      uint64_t r = key3(seed, 21, (uint64_t)g, 0);
      double dx = u01(r) - 0.5, dy = u01(mix64(r)) - 0.5;
      double t = ((double)x * dx + (double)y * dy) / 512.0;
      for (int c = 0; c < 3; ++c) col[c] += (u01(key3(seed, 22, (uint64_t)g, (uint64_t)c)) - 0.5) * 24.0 * t;
    }
    double a = vnoise(seed ^ 0xA1, x, y, 96);   /* pink weight */
    double b = vnoise(seed ^ 0xB2, x, y, 48);   /* purple weight */
    a = a > 0.45 ? (a - 0.45) * 1.6 : 0.0;
    b = b > 0.6 ? (b - 0.6) * 2.2 : 0.0;
    if (a + b > 1.0) { double s = a + b; a /= s; b /= s; }
    static const double pink[3] = {230.0, 150.0, 190.0}, purple[3] = {120.0, 80.0, 160.0};
    for (int c = 0; c < 3; ++c) {
      double v = col[c] * (1.0 - a - b) + pink[c] * a + purple[c] * b;
      v += 8.0 * gauss(key3(seed, 31, (uint64_t)(y * w + x), (uint64_t)c));
      row[3 * x + c] = (uint8_t)clampi(v, 0, 255);
    }
  }
}

/* ---------------------------------------------------------------- slide */
static int slide_is_tissue(uint64_t seed, int64_t x, int64_t y) {
  double f = 0.55 * vnoise(seed ^ 0x71, x, y, 4096) + 0.3 * vnoise(seed ^ 0x72, x, y, 1024) +
             0.15 * vnoise(seed ^ 0x73, x, y, 256);
  return f > 0.53;
}

static void slide_row(uint64_t seed, int64_t x0, int64_t y, int64_t w, uint8_t* row) {
  static const int64_t CELL = 24;
  for (int64_t i = 0; i < w; ++i) {
    int64_t x = x0 + i;
    double v[3];
    double sigma;
    if (!slide_is_tissue(seed, x, y)) {
      double base = 230.0 + 20.0 * vnoise(seed ^ 0x81, x, y, 2048);
      v[0] = base; v[1] = base - 2.0; v[2] = base + 1.0;
      sigma = 3.0;
    } else {
      double m = vnoise(seed ^ 0x91, x, y, 64);
      v[0] = 215.0 + 25.0 * m; v[1] = 120.0 + 40.0 * m; v[2] = 170.0 + 30.0 * m;
      int64_t cx = x / CELL, cy = y / CELL;
      for (int64_t gy = cy - 1; gy <= cy + 1; ++gy)
        for (int64_t gx = cx - 1; gx <= cx + 1; ++gx) {
          if (gx < 0 || gy < 0) continue;
          uint64_t r = key3(seed, 41, (uint64_t)gx, (uint64_t)gy);
          if ((r & 0xFF) >= 140) continue;                 /* ~55% of cells hold a nucleus */
          int64_t rad = 3 + (int64_t)((r >> 8) % 6);        /* radius 3..8 */
          int64_t ncx = gx * CELL + 4 + (int64_t)((r >> 16) % 16);
          int64_t ncy = gy * CELL + 4 + (int64_t)((r >> 24) % 16);
          int64_t dx = x - ncx, dy = y - ncy;
          if (dx * dx + dy * dy <= rad * rad) {
            double s = (double)((r >> 32) & 0xFF) / 255.0;
            v[0] = 80.0 + 30.0 * s; v[1] = 40.0 + 25.0 * s; v[2] = 120.0 + 30.0 * s;
          }
        }
      sigma = 10.0;
    }
    for (int c = 0; c < 3; ++c) {
      double n = sigma * gauss(key3(seed, 51, (uint64_t)(y * 1048576 + x), (uint64_t)c));
      row[3 * i + c] = (uint8_t)clampi(v[c] + n, 0, 255);
    }
  }
}

/* -------------------------------------------------------------- phantom */
typedef struct { double cx, cy, a, b, c, s, v; } ellipse_t;

static int phantom_ellipses(uint64_t seed, int64_t W, int64_t H, ellipse_t* e) {
  int n = 8 + (int)(mix64(seed ^ 0x61) % 9);   /* 8..16 */
  for (int k = 0; k < n; ++k) {
    uint64_t r0 = key3(seed, 61, (uint64_t)k, 0), r1 = key3(seed, 61, (uint64_t)k, 1), r2 = key3(seed, 61, (uint64_t)k, 2);
    e[k].cx = u01(r0) * (double)W;
    e[k].cy = u01(mix64(r0)) * (double)H;
    double m = (double)(W < H ? W : H);
    e[k].a = (0.05 + 0.3 * u01(r1)) * m;
    e[k].b = (0.05 + 0.3 * u01(mix64(r1))) * m;
    double dx = u01(r2) - 0.5, dy = u01(mix64(r2)) - 0.5;
    double nrm = sqrt(dx * dx + dy * dy);
    if (nrm < 1e-9) { dx = 1.0; dy = 0.0; nrm = 1.0; }
    e[k].c = dx / nrm; e[k].s = dy / nrm;
    e[k].v = 300.0 + 1800.0 * u01(mix64(mix64(r2)));
  }
  return n;
}

static void phantom_row(uint64_t seed, const ellipse_t* e, int n, int64_t x0, int64_t y, int64_t w, uint16_t* row) {
  for (int64_t i = 0; i < w; ++i) {
    int64_t x = x0 + i;
    double v = 60.0;
    for (int k = 0; k < n; ++k) {
      double dx = (double)x + 0.5 - e[k].cx, dy = (double)y + 0.5 - e[k].cy;
      double u = (dx * e[k].c + dy * e[k].s) / e[k].a, t = (-dx * e[k].s + dy * e[k].c) / e[k].b;
      double r2 = u * u + t * t;
      if (r2 < 1.0) v += e[k].v * (1.0 - r2);
    }
    if (v > 4095.0) v = 4095.0;
    const int64_t k = poisson(v, key3(seed, 71, (uint64_t)x, (uint64_t)y));
    row[i] = (uint16_t)(k > 4095 ? 4095 : k);
  }
}

/* ------------------------------------------------------------ threading */
typedef struct {
  int kind;
  uint64_t seed;
  int64_t x0, y0, w, h, W, H, pitch;
  uint8_t* out;
  int tid, nthreads;
  const ellipse_t* ell;
  int nell;
} job_t;

static void* run_job(void* arg) {
  job_t* j = (job_t*)arg;
  for (int64_t r = j->tid; r < j->h; r += j->nthreads) {
    uint8_t* row = j->out + r * j->pitch;
    if (j->kind == 0) stain_row(j->seed, j->y0 + r, j->w, row);
    else if (j->kind == 1) slide_row(j->seed, j->x0, j->y0 + r, j->w, row);
    else phantom_row(j->seed, j->ell, j->nell, j->x0, j->y0 + r, j->w, (uint16_t*)row);
  }
  return 0;
}

static void run(int kind, uint64_t seed, int64_t x0, int64_t y0, int64_t w, int64_t h, int64_t W, int64_t H,
                void* out, int64_t pitch, int threads) {
  ellipse_t ell[16];
  int nell = kind == 2 ? phantom_ellipses(seed, W, H, ell) : 0;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  pthread_t th[256];
  job_t jobs[256];
  for (int t = 0; t < threads; ++t) {
    job_t j = {kind, seed, x0, y0, w, h, W, H, pitch, (uint8_t*)out, t, threads, ell, nell};
    jobs[t] = j;
    if (threads > 1) pthread_create(&th[t], 0, run_job, &jobs[t]);
  }
  if (threads == 1) run_job(&jobs[0]);
  else for (int t = 0; t < threads; ++t) pthread_join(th[t], 0);
}

/* w x h tile, HWC uint8 rows of `pitch` bytes */
void isx_gen_stain(uint64_t seed, int64_t w, int64_t h, uint8_t* out, int64_t pitch, int threads) {
  run(0, seed, 0, 0, w, h, w, h, out, pitch, threads);
}
/* crop (x0, y0, w, h) of the slide image, HWC uint8 */
void isx_gen_slide(uint64_t seed, int64_t x0, int64_t y0, int64_t w, int64_t h, uint8_t* out, int64_t pitch, int threads) {
  run(1, seed, x0, y0, w, h, 0, 0, out, pitch, threads);
}
/* crop (x0, y0, w, h) of a W x H phantom image, uint16 */
void isx_gen_phantom(uint64_t seed, int64_t W, int64_t H, int64_t x0, int64_t y0, int64_t w, int64_t h,
                     uint16_t* out, int64_t pitch_bytes, int threads) {
  run(2, seed, x0, y0, w, h, W, H, out, pitch_bytes, threads);
}
uint64_t isx_gen_mix64(uint64_t x) { return mix64(x); }
/* the samplers, for their tests: n draws from the streams key0, key0 + 1, ... */
void isx_gen_normals(uint64_t key0, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = gauss(key0 + (uint64_t)i);
}
void isx_gen_poissons(double lam, uint64_t key0, int64_t n, int64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = poisson(lam, key0 + (uint64_t)i);
}
/* the series behind them: ln x, cos(2 pi u), ln k! */
void isx_gen_series(const double* x, const double* u, const int64_t* k, int64_t n, double* ln_x, double* cos_u, double* ln_k) {
  for (int64_t i = 0; i < n; ++i) {
    ln_x[i] = ln_d(x[i]);
    cos_u[i] = cos_2pi(u[i]);
    ln_k[i] = ln_fact(k[i]);
  }
}
