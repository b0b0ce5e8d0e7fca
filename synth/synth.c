/*
 * Seeded synthetic line lists (states + transitions) shaped like ExoMol
 * .states/.trans data (Sec. 2.3, Tables of the .states and .trans formats).
 *
 * This module produces INPUTS only.  It holds none of the method's arithmetic
 * (no partition function, intensity, profile or cross section) and is shared,
 * as data, by the FP64 oracle and the CUDA path.  Every random number comes from
 * a counter-based generator: the SplitMix64 output function (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied
 * to (seed, stream, counter), so any slice of a list can be regenerated
 * independently and the result does not depend on the thread count.
 *
 * Level schemes (readings of the workload descriptions, which leave these open):
 *  - diatomic: E(v,J) = 2000 v + 10 x - 1e-3 min(x, 5000)^2 with x = J(J+1)
 *    (clamped so the rotational energy keeps increasing past J ~ 70), or the
 *    literal quartic when `literal` is set; g = 3(2J+1); E_vib(v) = E(v, 0).
 *    State id = v * nJ + J.
 *  - polyatomic: three modes 1600/3650/3750 cm^-1 with v_i = 0..6, J = 0..99,
 *    k = 0..2J; E = sum_i omega_i v_i + 10 J(J+1)(1+u), u ~ U(-0.05, 0.05)
 *    per state; g = 2J+1; E_vib = sum_i omega_i v_i.  The 343*10000 level
 *    enumeration is repeated ("replicas", fresh u) until n_states, the last
 *    replica truncated.  State id = (r*343 + vib)*10000 + J*J + k.
 *  - transitions: lower state uniform over all states; dv uniform in {0,1,2}
 *    (on a uniformly drawn mode for polyatomics), dJ uniform in {-1,0,+1};
 *    redrawn up to 8 times while the upper state is out of range or
 *    (dv,dJ) = (0,0); after that dv = 0, dJ = -1 (or +1 at J = 0).
 *    A is log-uniform: A = 10^(a + (b-a) U).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
  z += GOLDEN;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Counter-based draw: stream separates independent uses of one seed. */
static inline uint64_t draw64(uint64_t seed, uint64_t stream, uint64_t ctr) {
  uint64_t base = sm64_mix(seed ^ (stream * 0xD1B54A32D192ED03ULL));
  return sm64_mix(base + ctr);
}

/* Uniform double in [0,1) from the top 53 bits. */
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

enum { ST_ENERGY = 1, ST_TRANS = 2, ST_A = 3, ST_GAMMA = 4, ST_NEXP = 5, ST_WEIGHT = 6 };

/* ---------------- diatomic ---------------- */

static double diatomic_erot(int64_t J, int literal) {
  double x = (double)J * (double)(J + 1);
  double xc = (!literal && x > 5000.0) ? 5000.0 : x;
  return 10.0 * x - 1e-3 * xc * xc;
}

void synth_states_diatomic(int64_t nv, int64_t nJ, int literal,
                           double* E, int32_t* g, double* E_vib) {
  int64_t n = nv * nJ;
#pragma omp parallel for schedule(static)
  for (int64_t id = 0; id < n; ++id) {
    int64_t v = id / nJ, J = id % nJ;
    E[id] = 2000.0 * (double)v + diatomic_erot(J, literal);
    g[id] = (int32_t)(3 * (2 * J + 1));
    if (E_vib) E_vib[id] = 2000.0 * (double)v;
  }
}

static int64_t diatomic_upper(uint64_t seed, int64_t t, int64_t lo, int64_t nv, int64_t nJ) {
  int64_t v = lo / nJ, J = lo % nJ;
  for (int tries = 0; tries < 8; ++tries) {
    uint64_t r = draw64(seed, ST_TRANS, (uint64_t)t * 64u + 1u + (uint64_t)tries);
    int dv = (int)((r >> 8) % 3u);
    int dJ = (int)((r >> 40) % 3u) - 1;
    if (dv == 0 && dJ == 0) continue;
    int64_t v2 = v + dv, J2 = J + dJ;
    if (v2 < 0 || v2 >= nv || J2 < 0 || J2 >= nJ) continue;
    return v2 * nJ + J2;
  }
  return v * nJ + (J > 0 ? J - 1 : J + 1);
}

void synth_transitions_diatomic(uint64_t seed, int64_t nv, int64_t nJ, int64_t t0, int64_t n,
                                double logA_lo, double logA_hi,
                                int32_t* upper, int32_t* lower, double* A64, float* A32) {
  int64_t ns = nv * nJ;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t t = t0 + i;
    int64_t lo = (int64_t)(u01(draw64(seed, ST_TRANS, (uint64_t)t * 64u)) * (double)ns);
    if (lo >= ns) lo = ns - 1;
    int64_t up = diatomic_upper(seed, t, lo, nv, nJ);
    upper[i] = (int32_t)up;
    lower[i] = (int32_t)lo;
    double ua = u01(draw64(seed, ST_A, (uint64_t)t));
    double a = pow(10.0, logA_lo + (logA_hi - logA_lo) * ua);
    if (A64) A64[i] = a;
    if (A32) A32[i] = (float)a;
  }
}

/* ---------------- polyatomic ---------------- */

#define PV 7          /* v_i = 0..6 */
#define NVIB (PV * PV * PV)
#define PJ 100        /* J = 0..99 */
#define NROT (PJ * PJ) /* sum_{J<100} (2J+1) */

static const double OMEGA[3] = {1600.0, 3650.0, 3750.0};

static void poly_decode(int64_t id, int64_t* r, int* v, int* J, int* k) {
  int64_t per = (int64_t)NVIB * NROT;
  *r = id / per;
  int64_t rem = id % per;
  int vib = (int)(rem / NROT);
  int rot = (int)(rem % NROT);
  v[0] = vib / (PV * PV); v[1] = (vib / PV) % PV; v[2] = vib % PV;
  int j = (int)floor(sqrt((double)rot));
  while (j * j > rot) --j;
  while ((j + 1) * (j + 1) <= rot) ++j;
  *J = j; *k = rot - j * j;
}

static int64_t poly_encode(int64_t r, const int* v, int J, int k) {
  int vib = (v[0] * PV + v[1]) * PV + v[2];
  return (r * NVIB + vib) * (int64_t)NROT + (int64_t)J * J + k;
}

void synth_states_polyatomic(uint64_t seed, int64_t id0, int64_t n, double* E, int32_t* g, double* E_vib) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t id = id0 + i, r; int v[3], J, k;
    poly_decode(id, &r, v, &J, &k);
    double ev = OMEGA[0] * v[0] + OMEGA[1] * v[1] + OMEGA[2] * v[2];
    double u = -0.05 + 0.1 * u01(draw64(seed, ST_ENERGY, (uint64_t)id));
    E[i] = ev + 10.0 * (double)J * (double)(J + 1) * (1.0 + u);
    g[i] = 2 * J + 1;
    if (E_vib) E_vib[i] = ev;
  }
}

void synth_transitions_polyatomic(uint64_t seed, int64_t n_states, int64_t t0, int64_t n,
                                  double logA_lo, double logA_hi,
                                  int32_t* upper, int32_t* lower, double* A64, float* A32) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t t = t0 + i;
    int64_t lo = (int64_t)(u01(draw64(seed, ST_TRANS, (uint64_t)t * 64u)) * (double)n_states);
    if (lo >= n_states) lo = n_states - 1;
    int64_t r; int v[3], J, k;
    poly_decode(lo, &r, v, &J, &k);
    int64_t up = -1;
    for (int tries = 0; tries < 8 && up < 0; ++tries) {
      uint64_t d = draw64(seed, ST_TRANS, (uint64_t)t * 64u + 1u + (uint64_t)tries);
      int dv = (int)((d >> 8) % 3u);
      int dJ = (int)((d >> 24) % 3u) - 1;
      int mode = (int)((d >> 40) % 3u);
      if (dv == 0 && dJ == 0) continue;
      int v2[3] = {v[0], v[1], v[2]};
      v2[mode] += dv;
      int J2 = J + dJ;
      if (v2[mode] >= PV || J2 < 0 || J2 >= PJ) continue;
      int k2 = (int)(u01(draw64(seed, ST_TRANS, (uint64_t)t * 64u + 16u + (uint64_t)tries)) * (double)(2 * J2 + 1));
      if (k2 > 2 * J2) k2 = 2 * J2;
      int64_t cand = poly_encode(r, v2, J2, k2);
      if (cand >= n_states) continue;
      up = cand;
    }
    if (up < 0) {
      int J2 = J > 0 ? J - 1 : J + 1;
      int k2 = k < 2 * J2 ? k : 2 * J2;
      up = poly_encode(r, v, J2, k2);
      if (up >= n_states) up = lo; /* degenerate: nu = 0, dropped downstream */
    }
    upper[i] = (int32_t)up;
    lower[i] = (int32_t)lo;
    double ua = u01(draw64(seed, ST_A, (uint64_t)t));
    double a = pow(10.0, logA_lo + (logA_hi - logA_lo) * ua);
    if (A64) A64[i] = a;
    if (A32) A32[i] = (float)a;
  }
}

/* ---------------- per-line broadening parameters and weights ---------------- */

void synth_uniform_f32(uint64_t seed, int stream, int64_t t0, int64_t n, double lo, double hi, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    out[i] = (float)(lo + (hi - lo) * u01(draw64(seed, (uint64_t)stream, (uint64_t)(t0 + i))));
}

/* Standard normal deviates by the Box-Muller transform, one pair of uniforms per value. */
void synth_normal_f32(uint64_t seed, int64_t n, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double u1 = u01(draw64(seed, ST_WEIGHT, (uint64_t)i * 2u));
    double u2 = u01(draw64(seed, ST_WEIGHT, (uint64_t)i * 2u + 1u));
    if (u1 < 1e-300) u1 = 1e-300;
    out[i] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

uint64_t synth_draw64(uint64_t seed, uint64_t stream, uint64_t ctr) { return draw64(seed, stream, ctr); }
