/*
 * Seeded synthetic input generators for the five SET workloads.
 *
 * Shared by the oracle tests, the GPU parity tests and bench.py: both sides of
 * every parity check read bytes produced here.  This file holds none of the
 * method's arithmetic (no stage of any pipeline); it only maps a counter-based
 * random stream onto the input distributions of each workload.
 *
 * Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  dg_rand(seed, i) is the i-th output
 * (0-based) of SplitMix64 started at state `seed`, so any element can be drawn
 * independently of the others.
 *
 * Compile with -ffp-contract=off so that the few floating-point mappings give
 * the same bytes on x86-64 and aarch64.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define DG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t dg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t dg_rand(uint64_t seed, uint64_t i) { return dg_mix(seed + (i + 1) * DG_GAMMA); }

/* Per-job seed: workload tag in the top byte so that streams never collide. */
uint64_t dg_job_seed(uint64_t master, uint32_t tag, uint64_t job) {
  return dg_rand(master ^ ((uint64_t)tag << 56) ^ job, 0);
}

/* Uniform byte: the top 8 bits. */
void dg_fill_u8(uint64_t seed, uint64_t off, uint8_t* out, size_t n) {
#pragma omp parallel for schedule(static) if (n > (1u << 22))
  for (size_t i = 0; i < n; ++i) out[i] = (uint8_t)(dg_rand(seed, off + i) >> 56);
}

/* Uniform float in [-2^e, 2^e): k * 2^(e-23) - 2^e with k the top 24 bits.
 * Every value is exact in fp32 (a 24-bit integer times a power of two). */
static inline float dg_unif_sym(uint64_t r, int e) {
  const float k = (float)(uint32_t)(r >> 40);
  return ldexpf(k, e - 23) - ldexpf(1.0f, e);
}

void dg_fill_unif_sym_f32(uint64_t seed, uint64_t off, int e, float* out, size_t n) {
#pragma omp parallel for schedule(static) if (n > (1u << 20))
  for (size_t i = 0; i < n; ++i) out[i] = dg_unif_sym(dg_rand(seed, off + i), e);
}

float dg_unif_sym_f32(uint64_t seed, uint64_t idx, int e) { return dg_unif_sym(dg_rand(seed, idx), e); }

/* Uniform double in [0, 1) from the top 53 bits. */
double dg_unif01(uint64_t seed, uint64_t idx) {
  return (double)(dg_rand(seed, idx) >> 11) * 0x1.0p-53;
}

/* Round-to-nearest-even from fp32 bits to bf16 bits (finite inputs). */
static inline uint16_t dg_f32_to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

/* Box-Muller normal (cosine branch), draws off+2i and off+2i+1 for element i,
 * scaled by `scale`, rounded double -> fp32 -> bf16 (both round-to-nearest-even). */
void dg_fill_normal_bf16(uint64_t seed, uint64_t off, double scale, uint16_t* out, size_t n) {
#pragma omp parallel for schedule(static) if (n > (1u << 20))
  for (size_t i = 0; i < n; ++i) {
    const double u1 = ((double)(dg_rand(seed, off + 2 * i) >> 11) + 1.0) * 0x1.0p-53; /* (0,1] */
    const double u2 = (double)(dg_rand(seed, off + 2 * i + 1) >> 11) * 0x1.0p-53;     /* [0,1) */
    const double v = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2) * scale;
    out[i] = dg_f32_to_bf16((float)v);
  }
}

/* Side length log-uniform on [lo, hi]: round(exp(ln lo + u ln(hi/lo))), clamped. */
int dg_logunif_side(uint64_t seed, uint64_t idx, int lo, int hi) {
  const double u = dg_unif01(seed, idx);
  double v = floor(exp(log((double)lo) + u * log((double)hi / (double)lo)) + 0.5);
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return (int)v;
}

/* Exponential inter-arrival gap with rate lambda (seconds): -ln(1-u)/lambda. */
double dg_exp_gap(uint64_t seed, uint64_t idx, double lambda) {
  return -log1p(-dg_unif01(seed, idx)) / lambda;
}

/* Uniform float in [lo, hi): lo + (hi - lo) * k * 2^-24 with k the top 24 bits,
 * evaluated in double and rounded once to fp32. */
void dg_fill_unif_range_f32(uint64_t seed, uint64_t off, double lo, double hi, float* out, size_t n) {
#pragma omp parallel for schedule(static) if (n > (1u << 20))
  for (size_t i = 0; i < n; ++i)
    out[i] = (float)(lo + (hi - lo) * ((double)(uint32_t)(dg_rand(seed, off + i) >> 40) * 0x1.0p-24));
}
