// Line-side kernels: Boltzmann table and partition function, intensity/gather
// pass, stable compaction, LSD radix sort by (nu bits, index), per-line
// preparation, segment binning and profile work items.
#include <atomic>
#include <cstdio>

#include "kernels.cuh"

namespace pxc {

static std::atomic<int64_t> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }


__device__ __forceinline__ void set_err(unsigned* err, unsigned bits) { atomicOr(err, bits); }

// Window of grid indices of a line (R8): ceil((nu - cut - nu_min)/dnu), floor((nu + cut - nu_min)/dnu),
// plain IEEE double with explicit rounding intrinsics so no contraction can change a tie.  On a
// wavelength grid (R21: lambda_i = lambda_min + i dlambda, nu_i = U / lambda_i) the points with
// |nu_i - nu| <= cut are those with U/(nu + cut) <= lambda_i <= U/(nu - cut):
// ceil((U/(nu + cut) - lambda_min)/dlambda) .. floor((U/(nu - cut) - lambda_min)/dlambda), the
// last point when nu <= cut.
// ceil(num / den) and floor(num / den) of the IEEE quotient without a division in almost every
// case: q = num * inv (inv = 1/den rounded) is within 2^-52 |q| of num / den, so when q is farther
// than 2^-51 |q| from the nearest integer the quotient has the same ceiling and floor; otherwise
// (an exact or near-integer quotient, num = 0) the rounded division decides.
__device__ __forceinline__ bool quotient_clear(double q) {
  return fabs(q - rint(q)) > 0x1p-51 * fabs(q);
}
__device__ __forceinline__ double ceil_div(double num, double den, double inv) {
  const double q = num * inv;
  return quotient_clear(q) ? ceil(q) : ceil(__ddiv_rn(num, den));
}
__device__ __forceinline__ double floor_div(double num, double den, double inv) {
  const double q = num * inv;
  return quotient_clear(q) ? floor(q) : floor(__ddiv_rn(num, den));
}

__device__ __forceinline__ bool exact_window(double nu, const GridP& gp, int64_t* lo, int64_t* hi) {
  double a, b;
  if (gp.wl_unit > 0.0) {
    a = ceil(__ddiv_rn(__dsub_rn(__ddiv_rn(gp.wl_unit, __dadd_rn(nu, gp.cut)), gp.nu_min), gp.dnu));
    b = __dsub_rn(nu, gp.cut) > 0.0
            ? floor(__ddiv_rn(__dsub_rn(__ddiv_rn(gp.wl_unit, __dsub_rn(nu, gp.cut)), gp.nu_min), gp.dnu))
            : (double)(gp.n - 1);
  } else {
    a = ceil_div(__dsub_rn(__dsub_rn(nu, gp.cut), gp.nu_min), gp.dnu, gp.inv_dnu);
    b = floor_div(__dsub_rn(__dadd_rn(nu, gp.cut), gp.nu_min), gp.dnu, gp.inv_dnu);
  }
  double top = (double)(gp.n - 1);
  if (!(b >= 0.0) || a > top || a > b) return false;
  *lo = a < 0.0 ? 0 : (int64_t)a;
  *hi = b > top ? gp.n - 1 : (int64_t)b;
  return true;
}

// Sort key of a kept line (nu > 0): its bit pattern (ascending nu, R11), or the complement on a
// wavelength grid (descending nu = ascending wavelength, R21); the stable sort breaks ties by index.
__device__ __forceinline__ uint64_t line_key(double nu, const GridP& gp) {
  const uint64_t b = (uint64_t)__double_as_longlong(nu);
  return gp.wl_unit > 0.0 ? ~b & 0x7fffffffffffffffull : b;
}
__device__ __forceinline__ double key_nu(uint64_t k, const GridP& gp) {
  return __longlong_as_double((long long)(gp.wl_unit > 0.0 ? ~k & 0x7fffffffffffffffull : k));
}

// v 2^-k, bit for bit as ldexp(v, -k): a multiplication by the exact power of two while 2^-k is a
// normal double (both are the correctly rounded product), ldexp itself otherwise.
__device__ __forceinline__ bool pow2_normal(int k) { return k >= -1000 && k <= 1022; }
__device__ __forceinline__ double pow2_scale(int k) {
  return pow2_normal(k) ? __longlong_as_double((long long)(1023 - k) << 52) : 0.0;
}
__device__ __forceinline__ double scale_by(double v, int k, double s) { return pow2_normal(k) ? v * s : ldexp(v, -k); }

__device__ __forceinline__ bool window_meets_grid(double nu, const GridP& gp) {
  if (gp.exact_bounds) return nu >= gp.nu_keep_lo && nu <= gp.nu_keep_hi;
  int64_t lo, hi;
  return exact_window(nu, gp, &lo, &hi);
}

// ------------------------------------------------------------------ block reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ K-Q: Boltzmann table and Q
// e^x for the Boltzmann factors by Tang's table-driven method (ACM TOMS 15 (1989) 144-157):
// x = (64 m + j) ln2/64 + r with |r| <= ln2/128, e^x = 2^m 2^(j/64) e^r, e^r - 1 from its degree-5
// Taylor polynomial (the first omitted term is below 2^-54 of e^r), 2^(j/64) from a table of the
// correctly rounded values (evaluated in 60-digit decimal arithmetic).  About half the FP64
// operations of exp(); within ~1 ulp.  |x| >= 700 (the under- and overflow ranges, NaN) uses exp().
__device__ const double kExp2J64[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0,
};

__device__ __forceinline__ double exp_tang(double x, const double* __restrict__ tab) {
  const long long xb = __double_as_longlong(x);
  if ((xb & 0x7fffffffffffffffll) >= 0x4085e00000000000ll) return exp(x);  // |x| >= 700 or NaN
  // n = x 64/ln2 rounded to the nearest integer: adding 1.5 2^52 leaves n in the low word
  const double tn = fma(x, 92.332482616893657, 0x1.8p52);                  // 64 / ln2
  const int ni = __double2loint(tn);
  const double n = tn - 0x1.8p52;
  const double r = fma(-n, 0x1.abc9e3b39803fp-62, fma(-n, 0x1.62e42fefa39efp-7, x));  // ln2/64, two parts
  const double q = r * fma(fma(fma(fma(r, 1.0 / 120.0, 1.0 / 24.0), r, 1.0 / 6.0), r, 0.5), r, 1.0);
  const double t = tab[ni & 63];
  const double v = fma(t, q, t);  // in [0.99, 1.99]
  return __longlong_as_double(__double_as_longlong(v) + ((long long)(ni >> 6) << 52));
}

// b_s = exp(-c2 E_s / T) (LTE, Eq. pf), exp(-c2 E_vib/T_vib - c2 E_rot/T_rot) (Eq. Q nlte 2T) or
// n_vib exp(-c2 E_rot / T_rot) (vibronic densities, Eq. Q nlte Nvib); per-block partial sums of
// g b, g b E_rot, g b E_vib and (cooling function) g b S in a fixed order.
__global__ void __launch_bounds__(kThreadsQ) k_boltzmann(const double* __restrict__ E, const int32_t* __restrict__ g,
                                                         const double* __restrict__ Ev,
                                                         const double* __restrict__ nvib, int64_t n,
                                                         const SlotP* __restrict__ slots, int nslot,
                                                         double2* __restrict__ srec, int64_t stride,
                                                         StateFast* __restrict__ sfast,
                                                         const double* __restrict__ Ssum,
                                                         double* __restrict__ qpart, unsigned* err) {
  __shared__ double red[kThreadsQ / 32][kQMoments];
  __shared__ double tab[64];
  if (threadIdx.x < 64) tab[threadIdx.x] = kExp2J64[threadIdx.x];
  __syncthreads();
  for (int sl = 0; sl < nslot; ++sl) {
    const SlotP sp = slots[sl];
    const bool two_t = sp.c2_Tv > 0.0;
    const bool dens = !two_t && nvib != nullptr;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
    unsigned bad = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
      double e = E[s];
      double b = 0.0;
      float lb = -INFINITY;
      // NaN / infinity from the exponent bits (integer tests, off the FP64 pipe)
      const unsigned long long eb = (unsigned long long)__double_as_longlong(e);
      const bool nonfinite = (eb & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
      if (nonfinite && (eb & 0x000fffffffffffffull)) {
        b = 0.0;  // NaN: an absent state (R15)
      } else if (nonfinite) {
        bad |= ERRB_NONFINITE;
      } else {
        double x, er = e, ev = 0.0, w = 1.0;
        if (two_t || dens) {
          ev = Ev[s];
          er = e - ev;
          if (!isfinite(ev)) bad |= ERRB_NONFINITE;
        }
        if (two_t) {
          x = -(ev * sp.c2_Tv) - er * sp.c2_T;
        } else if (dens) {
          // Eq. (F nlte Nvib): n_vib exp(-c2 E_rot / T_rot)
          w = nvib[s];
          if (!isfinite(w)) bad |= ERRB_NONFINITE;
          x = -er * sp.c2_T;
        } else {
          x = -e * sp.c2_T;
        }
        if (x > kExpMax) {
          bad |= ERRB_OVERFLOW;
        } else {
          b = w * exp_tang(x, tab);
          // log2 b for the FP32 rejection bound (its margin absorbs the FP32 rounding here)
          lb = dens ? (float)(x * 1.4426950408889634 + log2(w)) : (float)x * 1.44269504f;
          double term = (double)g[s] * b;
          q0 += term;
          q1 = fma(term, er, q1);                // times c2 / T^2 in k_qfinal: dQ/dT (or dQ/dT_rot)
          if (two_t) q2 = fma(term, ev, q2);     // times c2 / T_vib^2: dQ/dT_vib
          if (Ssum) q3 = fma(term, Ssum[s], q3);
        }
      }
      if (srec) srec[(int64_t)sl * stride + s] = make_double2(e, b);
      if (sfast) {
        StateFast r;
        r.E = e;
        r.b = b;
        r.g = (double)g[s];
        r.gf = (float)g[s];
        r.lb = lb;
        sfast[s] = r;
      }
    }
    if (bad) set_err(err, bad);
    q1 = warp_sum(q1); q0 = warp_sum(q0); q2 = warp_sum(q2); q3 = warp_sum(q3);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[w][0] = q0; red[w][1] = q1; red[w][2] = q2; red[w][3] = q3; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a[kQMoments] = {0.0, 0.0, 0.0, 0.0};
      for (int i = 0; i < kThreadsQ / 32; ++i)
        for (int m = 0; m < kQMoments; ++m) a[m] += red[i][m];
      double* o = qpart + ((int64_t)blockIdx.x * nslot + sl) * kQMoments;
      for (int m = 0; m < kQMoments; ++m) o[m] = a[m];
    }
    __syncthreads();
  }
}

// qres[sl] = {Q, dQ/dT (or dQ/dT_rot), dQ/dT_vib, 1/(8 pi c Q)}; W_out[sl] (if given) =
// (h c / 4 pi Q) sum_s g_s b_s S_s, the cooling function of Eq. (cf).
__global__ void k_qfinal(const double* __restrict__ qpart, int nblk, int nslot, const SlotP* __restrict__ slots,
                         double* __restrict__ qres, double* __restrict__ W_out) {
  __shared__ double red[32][kQMoments];
  int sl = blockIdx.x;
  double a[kQMoments] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double* o = qpart + ((int64_t)b * nslot + sl) * kQMoments;
    for (int m = 0; m < kQMoments; ++m) a[m] += o[m];
  }
  for (int m = 0; m < kQMoments; ++m) a[m] = warp_sum(a[m]);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int m = 0; m < kQMoments; ++m) red[w][m] = a[m];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[kQMoments] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
      for (int m = 0; m < kQMoments; ++m) t[m] += red[i][m];
    const SlotP sp = slots[sl];
    double* r = qres + sl * 4;
    r[0] = t[0];
    r[1] = t[1] * sp.c2_T / sp.T;                                 // dQ/dT (or dQ/dT_rot)
    r[2] = sp.c2_Tv > 0.0 ? t[2] * sp.c2_Tv / sp.T_vib : 0.0;      // dQ/dT_vib
    r[3] = 1.0 / (8.0 * kPi * kC * t[0]);
    if (W_out) W_out[sl] = kH * kC * t[3] / (4.0 * kPi * t[0]);
  }
}

void launch_boltzmann(const pxc_states* st, const SlotP* slots_dev, int nslot, double2* srec, int64_t srec_stride,
                      StateFast* sfast, double* qpart, double* qres, unsigned* err, cudaStream_t s,
                      const double* Ssum, double* W_out) {
  k_boltzmann<<<kQBlocks, kThreadsQ, 0, s>>>(st->E, st->g, st->E_vib, st->n_vib, st->n, slots_dev, nslot, srec,
                                             srec_stride, sfast, Ssum, qpart, err);
  k_qfinal<<<nslot, 1024, 0, s>>>(qpart, kQBlocks, nslot, slots_dev, qres, W_out);
  note_launches(2);
}

// ------------------------------------------------------------------ cooling function: per-state rates
// S[u] += A nu over every line u -> l with nu = E[u] - E[l] > 0 (FP64 atomics; the order of the
// additions, and so the last bits of S, depends on scheduling).  With them the cooling function of
// Eq. (cf) is W = (h c / 4 pi Q) sum_u g_u b_u S_u, one more moment of the state pass.
__global__ void __launch_bounds__(256) k_cool_rates(const int32_t* __restrict__ up, const int32_t* __restrict__ lo,
                                                    const void* __restrict__ Av, int A32, int64_t n,
                                                    const double* __restrict__ E, int64_t ns,
                                                    double* __restrict__ S, unsigned* err) {
  unsigned bad = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = __ldcs(up + t), l = __ldcs(lo + t);
    const double A = A32 ? (double)__ldcs((const float*)Av + t) : __ldcs((const double*)Av + t);
    if (u < 0 || u >= ns || l < 0 || l >= ns) { bad |= ERRB_ID; continue; }
    if (!isfinite(A)) { bad |= ERRB_NONFINITE; continue; }
    const double nu = __dsub_rn(E[u], E[l]);
    if (nu > 0.0) atomicAdd(S + u, A * nu);
  }
  if (bad) set_err(err, bad);
}

void launch_cool_rates(const pxc_transitions* tr, const pxc_states* st, double* S, unsigned* err, cudaStream_t s) {
  cudaMemsetAsync(S, 0, sizeof(double) * (size_t)(st->n > 0 ? st->n : 1), s);
  if (tr->n == 0) return;
  int64_t blocks = (tr->n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_cool_rates<<<(unsigned)blocks, 256, 0, s>>>(tr->upper, tr->lower, tr->A, tr->A_is_f32, tr->n, st->E, st->n, S,
                                                err);
  note_launches(1);
}

// ------------------------------------------------------------------ per-state energy codes
// Ordered 64-bit key of a double (monotone in the value for non-NaN inputs).
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// words[0] = max key(-E), words[1] = max key(E) over finite E (0: none), words[2] = max g.
__global__ void __launch_bounds__(256) k_state_range(const double* __restrict__ E, const int32_t* __restrict__ g,
                                                     int64_t n, unsigned long long* __restrict__ words) {
  unsigned long long kmin = 0, kmax = 0, gm = 0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const double e = E[s];
    if (isfinite(e)) {
      const unsigned long long a = dkey(-e), b = dkey(e);
      kmin = a > kmin ? a : kmin;
      kmax = b > kmax ? b : kmax;
    }
    const int32_t gv = g[s];
    const unsigned long long gg = gv > 0 ? (unsigned long long)gv : 0ull;
    gm = gg > gm ? gg : gm;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long v = __shfl_down_sync(0xffffffffu, kmin, o);
    kmin = v > kmin ? v : kmin;
    v = __shfl_down_sync(0xffffffffu, kmax, o);
    kmax = v > kmax ? v : kmax;
    v = __shfl_down_sync(0xffffffffu, gm, o);
    gm = v > gm ? v : gm;
  }
  if ((threadIdx.x & 31) == 0) {
    if (kmin) atomicMax(&words[0], kmin);
    if (kmax) atomicMax(&words[1], kmax);
    if (gm) atomicMax(&words[2], gm);
  }
}

__device__ __forceinline__ QuantHdr quant_header(const unsigned long long* words) {
  QuantHdr h{};
  const unsigned long long kmin = words[0], kmax = words[1];
  const double gmax = (double)(words[2] > 0 ? words[2] : 1ull);
  h.log2_gmax = (float)(log2(gmax) + 1e-6);
  if (!kmin || !kmax) return h;  // no finite energy
  const double emin = -dkey_inv(kmin), emax = dkey_inv(kmax);
  const double span = emax - emin;
  const double inv = span > 0.0 ? (double)(kCodeMax - 2) / span : 1.0;
  if (!isfinite(span) || !(inv > 0.0) || !isfinite(inv)) return h;
  h.Emin = emin;
  h.inv_res = inv;
  h.res_f = __double2float_ru(__ddiv_ru(1.0, inv));
  h.Emin_f = __double2float_rd(emin);
  h.enabled = isfinite(h.res_f) && h.res_f > 0.f && isfinite(h.Emin_f);
  return h;
}

// q = floor((E - Emin) inv_res) within one code of the exact value, which the bounds' slack of one
// code below and two above absorbs: E - Emin in FP64 (no cancellation), the scaling in FP32
// (relative error ~1e-7 of at most 4094 codes), so two FP64-pipe operations per state.  Energy
// spans beyond ~4e33 (FP32 would overflow) scale in FP64.
__device__ __forceinline__ int quant_code(double e, const QuantHdr& h, float inv_res_f) {
  const unsigned long long eb = (unsigned long long)__double_as_longlong(e);
  if (!h.enabled || (eb & 0x7ff0000000000000ull) == 0x7ff0000000000000ull) return kCodeNone;  // inf, NaN
  const float x = inv_res_f > 1e-30f ? floorf((float)(e - h.Emin) * inv_res_f)
                                     : (float)floor((e - h.Emin) * h.inv_res);
  return x < 0.f ? 0 : (x > (float)kCodeMax ? kCodeMax : (int)x);
}

// One thread per 64-bit word: the 12-bit codes of five consecutive states.
__global__ void __launch_bounds__(256) k_state_quant(const double* __restrict__ E, int64_t n,
                                                     const unsigned long long* __restrict__ words,
                                                     code_t* __restrict__ code, QuantHdr* __restrict__ hdr) {
  __shared__ QuantHdr hs;
  if (threadIdx.x == 0) hs = quant_header(words);  // once per CTA (FP64 division and log2)
  __syncthreads();
  const QuantHdr h = hs;
  const float inv_res_f = (float)h.inv_res;
  if (blockIdx.x == 0 && threadIdx.x == 0) *hdr = h;
  const int64_t nw = (n + 4) / 5;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    code_t word = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int64_t st = 5 * w + i;
      const int q = st < n ? quant_code(E[st], h, inv_res_f) : kCodeNone;
      word |= (code_t)q << (12 * i);
    }
    code[w] = word;
  }
}

void launch_state_codes(const pxc_states* st, code_t* code, unsigned long long* words, cudaStream_t s) {
  cudaMemsetAsync(words, 0, 3 * sizeof(unsigned long long), s);
  const int64_t n = st->n;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  QuantHdr* hdr = reinterpret_cast<QuantHdr*>(words + kQuantWords);
  k_state_range<<<(unsigned)blocks, 256, 0, s>>>(st->E, st->g, n, words);
  k_state_quant<<<(unsigned)blocks, 256, 0, s>>>(st->E, n, words, code, hdr);
  note_launches(2);
}

// ------------------------------------------------------------------ K-I: intensities
// nu = E[u] - E[l] (FP64), keep = nu > 0 and window meets the grid and I >= threshold;
// I = g_u A (b_l - b_u) / (8 pi c nu^2 Q), the Boltzmann factors from the per-state table
// (b_l - b_u = e^{-c2 E''/T}(1 - e^{-c2 nu/T}) for LTE, and the Treanor form of Eq.
// (nlte ab 2T) for two temperatures since b_u/b_l = e^{-c2(nu_vib/T_vib + nu_rot/T_rot)}).
__global__ void __launch_bounds__(kThreadsI) k_lines(const int32_t* __restrict__ up, const int32_t* __restrict__ lo,
                                                     const void* __restrict__ Av, int A32, int64_t n,
                                                     const double2* __restrict__ srec, const int32_t* __restrict__ g,
                                                     int64_t ns, const double* __restrict__ qres, GridP gp,
                                                     BoundP bp, int use_grid, double threshold, int with_I,
                                                     uint64_t* __restrict__ key, double* __restrict__ Iv,
                                                     double* __restrict__ nu_out, uint32_t* __restrict__ bcount,
                                                     unsigned long long* __restrict__ maxbits, unsigned* err) {
  __shared__ uint32_t wk[kThreadsI / 32];
  __shared__ unsigned long long wm[kThreadsI / 32];
  const double invQ = with_I ? qres[3] : 0.0;
  const int64_t base = (int64_t)blockIdx.x * kLinesPerBlockI;
  uint32_t kept = 0;
  unsigned long long mx = 0;
  unsigned bad = 0;
#pragma unroll 2
  for (int k = 0; k < kLinesPerBlockI / kThreadsI; ++k) {
    int64_t t = base + k * kThreadsI + threadIdx.x;
    if (t >= n) break;
    int64_t u = up[t], l = lo[t];
    double A = A32 ? (double)((const float*)Av)[t] : ((const double*)Av)[t];
    uint64_t kk = kSentinelKey;
    double I = 0.0;
    double nu = __longlong_as_double(0x7ff8000000000000ll);
    if (u < 0 || u >= ns || l < 0 || l >= ns) {
      bad |= ERRB_ID;
    } else {
      if (!isfinite(A)) bad |= ERRB_NONFINITE;
      double2 ru = srec[u], rl = srec[l];
      nu = __dsub_rn(ru.x, rl.x);
      bool keep = nu > 0.0;
      if (keep && use_grid) keep = window_meets_grid(nu, gp);
      if (keep && with_I) {
        // |I| >= threshold tested as |num| >= threshold * den (no division for dropped lines)
        double num, den;
        line_value(bp.mode, bp.c2_Td, (double)g[u], A, invQ, rl.y, ru.y, nu, &num, &den);
        keep = fabs(num) >= threshold * den;
        if (keep) I = num / den;
      }
      if (keep) {
        kk = line_key(nu, gp);
        ++kept;
        unsigned long long ib = (unsigned long long)__double_as_longlong(fabs(I));
        mx = ib > mx ? ib : mx;
      } else {
        I = 0.0;
      }
    }
    key[t] = kk;
    if (with_I) Iv[t] = I;
    if (nu_out) nu_out[t] = nu;
  }
  if (bad) set_err(err, bad);
  kept = warp_sum(kept);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long v = __shfl_down_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { wk[w] = kept; wm[w] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    unsigned long long m = 0;
    for (int i = 0; i < kThreadsI / 32; ++i) { s += wk[i]; m = wm[i] > m ? wm[i] : m; }
    bcount[blockIdx.x] = s;
    if (with_I && m) atomicMax(maxbits, m);
  }
}

void launch_lines(const pxc_transitions* tr, const int32_t* g, int64_t ns, const double2* srec,
                  const double* qres, const GridP& gp, const BoundP& bp, int use_grid, double threshold,
                  int with_intensity,
                  uint64_t* key, double* Iv, double* nu_out, uint32_t* bcount, int64_t nblk,
                  unsigned long long* maxbits, unsigned* err, cudaStream_t s) {
  if (nblk == 0) return;
  k_lines<<<(unsigned)nblk, kThreadsI, 0, s>>>(tr->upper, tr->lower, tr->A, tr->A_is_f32, tr->n, srec, g, ns, qres,
                                               gp, bp, use_grid, threshold, with_intensity, key, Iv, nu_out, bcount,
                                               maxbits, err);
  note_launches(1);
}

// ------------------------------------------------------------------ K-I, compacting form (cross sections)
// Same selection as k_lines, but kept lines are written compacted per block in index order
// (key, index) and I by transition index; rejected lines write nothing.  With a threshold,
// a conservative FP32 upper bound on |I| rejects lines without touching the FP64 Boltzmann
// table or dividing: |I| <= g_u A max(b_l, b_u) m / (8 pi c Q nu^2), m = min(1, c2 nu/T) for
// LTE (b_l - b_u = b_l (1 - e^{-c2 nu/T})) and m = 1 for two temperatures, evaluated in log2
// units with a 1e-3 margin that covers every FP32 rounding in it.
//
// Before any 32-byte state record is read, a prefilter on the 12-bit state codes (1.6 bytes per
// state, 80 MB for 5e7 states, about half of it found in L2) rejects lines whose nu is
// certainly outside the kept window, and, for LTE with a threshold, lines whose intensity is
// certainly below it: nu_lo = (d - 3) res, nu_hi = (d + 3) res with d = q_u - q_l, b_l <=
// exp(-c2 E_lo(q_l) / T), g_u <= max g.  Only the surviving candidates gather their states.


// Block-wide exclusive rank of `flag` among the 256 threads in thread order, and the total.
__device__ __forceinline__ uint32_t block_rank(bool flag, uint32_t* wsum, uint32_t* total) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  uint32_t before = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kThreadsI / 32; ++i) { before += i < w ? wsum[i] : 0u; tot += wsum[i]; }
  __syncthreads();
  *total = tot;
  return before + __popc(m & ((1u << lane) - 1u));
}

// 12-bit code of state s: one 8-byte load of its word (kept in L2 with the evict-last policy: the
// state codes are re-read at random), then the code's 12 bits.
__device__ __forceinline__ int ld_code(const code_t* tab, int32_t s, uint64_t pol) {
  const unsigned su = (unsigned)s, w = su / 5u;
  unsigned long long v;
  asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(tab + w), "l"(pol));
  return (int)(v >> (12u * (su - 5u * w))) & 0xfff;
}

// Per-block constants of the compacting intensity pass (computed once per CTA by one thread).
struct LinesConst {
  double invQ;
  float l2invQ, lo_scale, hi_scale, Emin_f, log2_gmax;
  int dlo, dhi, pre, pre_thr;
};

__device__ LinesConst lines_const(const code_t* code, const QuantHdr* qhp, const double* qres, const GridP& gp,
                                  double threshold, const BoundP& bp, int with_I) {
  LinesConst c{};
  c.invQ = with_I ? qres[3] : 0.0;
  c.l2invQ = with_I ? (float)log2(c.invQ) : 0.f;
  QuantHdr qh{};
  if (code) qh = *qhp;
  const double wl = gp.exact_bounds ? gp.nu_keep_lo : gp.nu_span_lo;
  const double wh = gp.exact_bounds ? gp.nu_keep_hi : gp.nu_span_hi;
  // the codes are used when their resolution is at most 1/16 of the kept nu range (a list
  // whose energies span far more than the window gains nothing from them)
  c.pre = code != nullptr && qh.enabled && (wh - wl) * qh.inv_res >= 16.0;
  // the code bound on b_l holds for LTE absorption only
  c.pre_thr = c.pre && with_I && threshold > 0.0 && bp.lte && bp.mode == IMODE_ABS;
  c.dlo = INT_MIN;
  c.dhi = INT_MAX;
  if (c.pre) {
    // kept lines have nu in [wl, wh] (infinite ends: none kept); widen by two grid steps,
    // a relative 1e-9 and four code steps
    const double a = isinf(wl) ? (wl > 0 ? 2e9 : -2e9)
                               : floor((wl - 2.0 * gp.dnu - 1e-9 * fabs(wl)) * qh.inv_res) - 4.0;
    const double b = isinf(wh) ? (wh > 0 ? 2e9 : -2e9)
                               : ceil((wh + 2.0 * gp.dnu + 1e-9 * fabs(wh)) * qh.inv_res) + 4.0;
    c.dlo = a < -1e9 ? -1000000000 : (a > 1e9 ? 1000000000 : (int)a);
    c.dhi = b > 1e9 ? 1000000000 : (b < -1e9 ? -1000000000 : (int)b);
  }
  c.lo_scale = qh.res_f * 0.99999f;
  c.hi_scale = qh.res_f * 1.00001f;
  c.Emin_f = qh.Emin_f;
  c.log2_gmax = qh.log2_gmax;
  return c;
}

// One line's inputs as streamed: upper and lower ids and the bit pattern of A (FP32 or FP64).
struct LineIn {
  int32_t u, l;
  unsigned long long ab;
};

__device__ __forceinline__ LineIn line_load(int64_t t, const int32_t* __restrict__ up, const int32_t* __restrict__ lo,
                                            const void* __restrict__ Av, int A32) {
  LineIn x;
  x.u = __ldcs(up + t);
  x.l = __ldcs(lo + t);
  x.ab = A32 ? (unsigned long long)__float_as_uint(__ldcs((const float*)Av + t))
             : (unsigned long long)__double_as_longlong(__ldcs((const double*)Av + t));
  return x;
}

// Whether a loaded line is a candidate: valid ids and, when the codes are on, a code-bound nu inside
// the kept window and (LTE with a threshold) a code bound on |I| at or above the threshold.  Bad ids
// and non-finite A are reported in `bad`.
__device__ __forceinline__ bool line_test(const LineIn& x, int A32, int64_t ns, const code_t* __restrict__ code,
                                          const LinesConst& c, const BoundP& bp, uint64_t pol, unsigned* bad) {
  const int32_t u = x.u, l = x.l;
  const bool finite = A32 ? (x.ab & 0x7f800000ull) != 0x7f800000ull
                          : (x.ab & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
  // ids in [0, ns): one unsigned comparison each (state counts are below 2^31)
  if ((unsigned)u >= (unsigned)ns || (unsigned)l >= (unsigned)ns) {
    *bad |= ERRB_ID;
    return false;
  }
  if (!finite) *bad |= ERRB_NONFINITE;
  if (!c.pre) return true;
  const int qu = ld_code(code, u, pol), ql = ld_code(code, l, pol);
  if (qu == kCodeNone || ql == kCodeNone) return true;
  const int d = qu - ql;
  if (d < c.dlo || d > c.dhi) return false;
  if (c.pre_thr && d > 3) {
    const float Af = A32 ? __uint_as_float((unsigned)x.ab) : (float)__longlong_as_double((long long)x.ab);
    const float kl2e = 1.4426950408889634f;
    const float nul = (float)(d - 3) * c.lo_scale, nuh = (float)(d + 3) * c.hi_scale;
    const float m = fminf(1.f, bp.c2_T * nuh);
    const float Elo = fmaf((float)(ql - 1), ql >= 1 ? c.lo_scale : c.hi_scale, c.Emin_f);
    const float lbl = -(bp.c2_T * kl2e) * Elo;  // log2 of the upper bound of b_l
    const float Pb = Af * m / (nul * nul);
    if (__log2f(Pb) + c.log2_gmax + lbl + c.l2invQ < bp.log2_thr - 1e-6f * fabsf(lbl)) return false;
  }
  return true;
}

// The intensity pass of the cross-section path in two kernels.  The prefilter streams the lines
// (one warp per unit of kUnitLines consecutive lines) and writes each unit's candidates, in line
// order, to the unit's range of three candidate arrays; it holds few registers, so the random
// code gathers it waits on have the whole SM's worth of warps in flight.  The exact pass then
// takes each unit's candidates 32 at a time on full warps: the 32-byte state records, exact nu and
// window, the FP32 bound with the exact log2 b, then the FP64 test |num| >= S_min nu^2 and
// I = num / nu^2; kept lines go to the unit's staging range in line order, counted per unit.
// When the codes are off (a list whose energies span far more than the kept window) the exact
// pass reads the lines directly and the prefilter does nothing.
__global__ void __launch_bounds__(kThreadsI, 8) k_lines_pre(const int32_t* __restrict__ up,
                                                         const int32_t* __restrict__ lo,
                                                         const void* __restrict__ Av, int A32, int64_t n,
                                                         const code_t* __restrict__ code,
                                                         const QuantHdr* __restrict__ qhp, int64_t ns,
                                                         const double* __restrict__ qres, GridP gp, double threshold,
                                                         BoundP bp, int with_I, uint32_t* __restrict__ cand_t,
                                                         uint64_t* __restrict__ cand_ul, uint64_t* __restrict__ cand_a,
                                                         uint32_t* __restrict__ ccount, int64_t nunit, unsigned* err) {
  __shared__ LinesConst kc;
  if (threadIdx.x == 0) kc = lines_const(code, qhp, qres, gp, threshold, bp, with_I);
  __syncthreads();
  const LinesConst c = kc;
  if (!c.pre) return;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t unit = (int64_t)blockIdx.x * (kThreadsI / 32) + (threadIdx.x >> 5);
  if (unit >= nunit) return;
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  const int64_t ubase = unit * kUnitLines;
  unsigned bad = 0;
  uint32_t nb = 0;
  // the next round's line arrays are requested before this round's code gathers, so the two
  // memory latencies of a round overlap
  LineIn nx{0, 0, 0ull};
  if (ubase + lane < n) nx = line_load(ubase + lane, up, lo, Av, A32);
  for (int r = 0; r < kUnitLines / 32; ++r) {
    const int64_t t = ubase + r * 32 + lane;
    const LineIn x = nx;
    if (r + 1 < kUnitLines / 32 && t + 32 < n) nx = line_load(t + 32, up, lo, Av, A32);
    const bool cand = t < n && line_test(x, A32, ns, code, c, bp, pol, &bad);
    const unsigned cm = __ballot_sync(0xffffffffu, cand);
    if (cand) {
      const int64_t o = ubase + nb + __popc(cm & lt);
      cand_t[o] = (uint32_t)t;
      cand_ul[o] = ((uint64_t)(uint32_t)x.u << 32) | (uint32_t)x.l;
      cand_a[o] = x.ab;
    }
    nb += __popc(cm);
  }
  if (lane == 0) ccount[unit] = nb;
  if (bad) set_err(err, bad);
}

__global__ void __launch_bounds__(kThreadsI) k_lines_exact(const int32_t* __restrict__ up,
                                                           const int32_t* __restrict__ lo,
                                                           const void* __restrict__ Av, int A32, int64_t n,
                                                           const code_t* __restrict__ code,
                                                           const QuantHdr* __restrict__ qhp,
                                                           const StateFast* __restrict__ sfast, int64_t ns,
                                                           const double* __restrict__ qres, GridP gp,
                                                           double threshold, BoundP bp, int with_I,
                                                           const uint32_t* __restrict__ cand_t,
                                                           const uint64_t* __restrict__ cand_ul,
                                                           const uint64_t* __restrict__ cand_a,
                                                           const uint32_t* __restrict__ ccount,
                                                           uint64_t* __restrict__ kstage, uint32_t* __restrict__ istage,
                                                           double* __restrict__ Iv, uint32_t* __restrict__ ucount,
                                                           int64_t nunit, unsigned long long* __restrict__ maxbits,
                                                           unsigned* err) {
  constexpr int NW = kThreadsI / 32;
  __shared__ LinesConst kc;
  if (threadIdx.x == 0) kc = lines_const(code, qhp, qres, gp, threshold, bp, with_I);
  __syncthreads();
  const LinesConst c = kc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t unit = (int64_t)blockIdx.x * NW + warp;
  const long long lo_bits = __double_as_longlong(gp.nu_keep_lo), hi_bits = __double_as_longlong(gp.nu_keep_hi);
  unsigned long long mx = 0;
  unsigned bad = 0;
  uint32_t run = 0;  // kept lines of this unit so far
  const int64_t ubase = unit * kUnitLines;
  if (unit < nunit) {
    // candidates of this unit: from the prefilter, or every line when the codes are off
    const int64_t ncand = c.pre ? (int64_t)ccount[unit] : min((int64_t)kUnitLines, n - ubase);
    for (int64_t j0 = 0; j0 < ncand; j0 += 32) {
      bool keep = false;
      double nu = 0.0, I = 0.0;
      uint32_t t = 0;
      if (j0 + lane < ncand) {
        int32_t u, l;
        unsigned long long ab;
        bool ok = true;
        if (c.pre) {
          const int64_t o = ubase + j0 + lane;
          t = cand_t[o];
          const uint64_t ul = cand_ul[o];
          u = (int32_t)(ul >> 32);
          l = (int32_t)(uint32_t)ul;
          ab = cand_a[o];
        } else {
          t = (uint32_t)(ubase + j0 + lane);
          const LineIn x = line_load(t, up, lo, Av, A32);
          ok = line_test(x, A32, ns, nullptr, c, bp, 0, &bad);
          u = x.u;
          l = x.l;
          ab = x.ab;
        }
        if (ok) {
          const double A = A32 ? (double)__uint_as_float((unsigned)ab) : __longlong_as_double((long long)ab);
          const float Af = A32 ? __uint_as_float((unsigned)ab) : (float)A;
          const StateFast fu = sfast[u], fl = sfast[l];
          nu = __dsub_rn(fu.E, fl.E);
          if (gp.exact_bounds) {
            const long long nbits = __double_as_longlong(nu);
            keep = nbits >= lo_bits && nbits <= hi_bits;
          } else {
            int64_t a, b;
            keep = nu > 0.0 && exact_window(nu, gp, &a, &b);
          }
          if (keep && with_I) {
            if (threshold > 0.0) {
              // conservative FP32 log2 bound on |value| (see line_value)
              const float nuf = (float)nu;
              float P, lbb;
              if (bp.mode == IMODE_EMISSION) {
                P = fu.gf * Af * nuf * (float)kTwoHC2;
                lbb = fu.lb;
              } else {
                const float m = bp.lte ? fminf(1.f, bp.c2_T * nuf) : 1.f;
                P = fu.gf * Af * m / (nuf * nuf);
                lbb = fmaxf(fu.lb, fl.lb);
              }
              if (__log2f(P) + lbb + c.l2invQ < bp.log2_thr) keep = false;
            }
            if (keep) {
              double num, den;
              line_value(bp.mode, bp.c2_Td, fu.g, A, c.invQ, fl.b, fu.b, nu, &num, &den);
              keep = fabs(num) >= threshold * den;
              if (keep) I = num / den;
            }
          }
        }
      }
      const unsigned kb = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int64_t o = ubase + run + __popc(kb & lt);
        kstage[o] = line_key(nu, gp);
        istage[o] = t;
        if (with_I) {
          Iv[t] = I;
          const unsigned long long ib = (unsigned long long)__double_as_longlong(fabs(I));
          mx = ib > mx ? ib : mx;
        }
      }
      run += __popc(kb);
    }
    if (lane == 0) ucount[unit] = run;
  }
  if (bad) set_err(err, bad);
  if (with_I) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_down_sync(0xffffffffu, mx, o);
      mx = v > mx ? v : mx;
    }
    // one atomic per warp (no block barrier: a warp that finishes early frees its slot at once)
    if (lane == 0 && mx) atomicMax(maxbits, mx);
  }
}

void launch_lines_compact(const pxc_transitions* tr, int64_t ns, const code_t* code, const QuantHdr* qh,
                          const StateFast* sfast,
                          const double* qres, const GridP& gp, double threshold, const BoundP& bp, int with_I,
                          uint32_t* cand_t, uint64_t* cand_ul, uint64_t* cand_a, uint32_t* ccount,
                          uint64_t* kstage, uint32_t* istage, double* Iv, uint32_t* ucount, int64_t nunit,
                          unsigned long long* maxbits, unsigned* err, cudaStream_t s) {
  if (nunit == 0) return;
  const int64_t nblk = (nunit + kThreadsI / 32 - 1) / (kThreadsI / 32);
  k_lines_pre<<<(unsigned)nblk, kThreadsI, 0, s>>>(tr->upper, tr->lower, tr->A, tr->A_is_f32, tr->n, code, qh, ns,
                                                   qres, gp, threshold, bp, with_I, cand_t, cand_ul, cand_a, ccount,
                                                   nunit, err);
  k_lines_exact<<<(unsigned)nblk, kThreadsI, 0, s>>>(tr->upper, tr->lower, tr->A, tr->A_is_f32, tr->n, code, qh,
                                                     sfast, ns, qres, gp, threshold, bp, with_I, cand_t, cand_ul,
                                                     cand_a, ccount, kstage, istage, Iv, ucount, nunit, maxbits, err);
  note_launches(2);
}

// Copies each unit's staged kept lines to its offset (exclusive scan of the counts, total at
// [nunit]); one warp per unit.
__global__ void __launch_bounds__(256) k_compact_staged(const uint64_t* __restrict__ kstage,
                                                        const uint32_t* __restrict__ istage,
                                                        const uint32_t* __restrict__ uoff, int64_t nunit,
                                                        uint64_t* __restrict__ okey, uint32_t* __restrict__ oidx) {
  const int64_t u = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (u >= nunit) return;
  const uint32_t off = uoff[u], cnt = uoff[u + 1] - off;
  const int64_t base = u * kUnitLines;
  for (uint32_t r = threadIdx.x & 31; r < cnt; r += 32) {
    okey[off + r] = kstage[base + r];
    oidx[off + r] = istage[base + r];
  }
}

void launch_compact_staged(const uint64_t* kstage, const uint32_t* istage, const uint32_t* uoff, int64_t nunit,
                           uint64_t* okey, uint32_t* oidx, cudaStream_t s) {
  if (nunit == 0) return;
  k_compact_staged<<<(unsigned)((nunit + 7) / 8), 256, 0, s>>>(kstage, istage, uoff, nunit, okey, oidx);
  note_launches(1);
}

// ------------------------------------------------------------------ exclusive scan of block counts (one CTA)
// In-place exclusive scan of n counts (16-byte aligned) by one CTA of 1024 threads, total at [n] and in *total:
// tiles of 4096 counts, each thread four consecutive ones (one 16-byte load and store), a warp
// scan and a scan of the 32 warp totals, the running carry between tiles.
__global__ void __launch_bounds__(1024) k_scan_counts(uint32_t* __restrict__ c, int64_t n,
                                                      unsigned long long* total) {
  __shared__ unsigned long long wsum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned long long carry = 0;
  for (int64_t base = 0; base < n; base += 4096) {
    const int64_t i0 = base + 4 * (int64_t)t;
    uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if (i0 + 3 < n) {
      const uint4 q = *reinterpret_cast<const uint4*>(c + i0);
      v0 = q.x; v1 = q.y; v2 = q.z; v3 = q.w;
    } else {
      if (i0 < n) v0 = c[i0];
      if (i0 + 1 < n) v1 = c[i0 + 1];
      if (i0 + 2 < n) v2 = c[i0 + 2];
    }
    const unsigned long long sum = (unsigned long long)v0 + v1 + v2 + v3;
    unsigned long long x = sum;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long y = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += z;
      }
      wsum[lane] = y;
    }
    __syncthreads();
    const unsigned long long e0 = carry + (w ? wsum[w - 1] : 0ull) + x - sum;
    const unsigned long long e1 = e0 + v0, e2 = e1 + v1, e3 = e2 + v2;
    if (i0 + 3 < n) {
      *reinterpret_cast<uint4*>(c + i0) = make_uint4((uint32_t)e0, (uint32_t)e1, (uint32_t)e2, (uint32_t)e3);
    } else {
      if (i0 < n) c[i0] = (uint32_t)e0;
      if (i0 + 1 < n) c[i0 + 1] = (uint32_t)e1;
      if (i0 + 2 < n) c[i0 + 2] = (uint32_t)e2;
    }
    carry += wsum[31];
    __syncthreads();  // wsum is rewritten by the next tile
  }
  if (t == 0) {
    *total = carry;
    c[n] = (uint32_t)carry;
  }
}

void launch_scan_counts(uint32_t* bcount, int64_t nblk, unsigned long long* total, cudaStream_t s) {
  k_scan_counts<<<1, 1024, 0, s>>>(bcount, nblk, total);
  note_launches(1);
}


// ------------------------------------------------------------------ non-zero lines of one temperature
// Stable compaction of the sorted lines whose FP32 scaled intensity is non-zero (their records and
// intensities), for the batched call: lines far below a list's strongest line round to zero at low
// temperatures and add nothing to sigma.  Blocks of 256 threads take kUnitLines consecutive lines
// each (count, exclusive scan of the counts, then writes in line order).
__global__ void __launch_bounds__(256) k_nz_count(const float* __restrict__ Is, const unsigned long long* __restrict__ n_dev,
                                                  uint32_t* __restrict__ bcount) {
  __shared__ uint32_t wsum[8];
  const int64_t n = (int64_t)*n_dev;
  const int64_t base = (int64_t)blockIdx.x * kUnitLines;
  uint32_t c = 0;
  for (int r = 0; r < kUnitLines / 256; ++r) {
    const int64_t j = base + r * 256 + threadIdx.x;
    c += (j < n && Is[j] != 0.f) ? 1u : 0u;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int i = 0; i < 8; ++i) t += wsum[i];
    bcount[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_nz_write(const int4* __restrict__ pos, const float2* __restrict__ par,
                                                  const float* __restrict__ Is, const unsigned long long* __restrict__ n_dev,
                                                  const uint32_t* __restrict__ boff, int4* __restrict__ pos_c,
                                                  float2* __restrict__ par_c, float* __restrict__ Is_c) {
  __shared__ uint32_t wsum[8];
  const int64_t n = (int64_t)*n_dev;
  const int64_t base = (int64_t)blockIdx.x * kUnitLines;
  if (base >= n) return;  // uniform per block
  int64_t o = boff[blockIdx.x];
  for (int r = 0; r < kUnitLines / 256; ++r) {
    const int64_t j = base + r * 256 + threadIdx.x;
    const float v = j < n ? Is[j] : 0.f;
    uint32_t tot;
    const uint32_t rank = block_rank(v != 0.f, wsum, &tot);
    if (v != 0.f) {
      pos_c[o + rank] = pos[j];
      par_c[o + rank] = par[j];
      Is_c[o + rank] = v;
    }
    o += tot;
  }
}

void launch_compact_nonzero(const int4* pos, const float2* par, const float* Is, const unsigned long long* n_dev,
                            int64_t n_max, uint32_t* bcount, unsigned long long* nnz_dev, int4* pos_c, float2* par_c,
                            float* Is_c, cudaStream_t s) {
  const int64_t nblk = (n_max + kUnitLines - 1) / kUnitLines;
  if (nblk == 0) {
    cudaMemsetAsync(nnz_dev, 0, sizeof(unsigned long long), s);
    return;
  }
  k_nz_count<<<(unsigned)nblk, 256, 0, s>>>(Is, n_dev, bcount);
  k_scan_counts<<<1, 1024, 0, s>>>(bcount, nblk, nnz_dev);
  k_nz_write<<<(unsigned)nblk, 256, 0, s>>>(pos, par, Is, n_dev, bcount, pos_c, par_c, Is_c);
  note_launches(3);
}

// ------------------------------------------------------------------ LSD radix sort, 8 passes of 8 bits
// Pass: per-tile digit histogram -> per-digit exclusive scan over tiles -> stable scatter.
// Per-tile digit histograms.  The grid is sized for the largest list; the CTAs stride over the
// tiles the kept count actually fills (n is only known on the device).
__global__ void __launch_bounds__(kSortThreads) k_hist(const uint64_t* __restrict__ key,
                                                       const unsigned long long* __restrict__ n_dev, int64_t nblk,
                                                       int shift, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t h[256];
  const int64_t n = (int64_t)*n_dev;
  const int64_t act = (n + kSortTile - 1) / kSortTile;
  for (int64_t t = blockIdx.x; t < act; t += gridDim.x) {
    const int64_t base = t * kSortTile;
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int i = 0; i < kSortItems; ++i) {
      int64_t j = base + i * kSortThreads + threadIdx.x;
      if (j < n) atomicAdd(&h[(unsigned)(key[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    cnt[(int64_t)threadIdx.x * nblk + t] = h[threadIdx.x];
    __syncthreads();
  }
}

// One CTA per digit: exclusive scan of that digit's row over the active tiles; row total at the end.
__global__ void k_rowscan(uint32_t* __restrict__ cnt, const unsigned long long* __restrict__ n_dev, int64_t nblk,
                          uint32_t* __restrict__ rowtot) {
  __shared__ uint32_t part[1024];
  const int64_t n = (int64_t)*n_dev;
  const int64_t act = (n + kSortTile - 1) / kSortTile;
  uint32_t* row = cnt + (int64_t)blockIdx.x * nblk;
  int64_t per = (act + blockDim.x - 1) / blockDim.x;
  int64_t a = threadIdx.x * per, b = a + per < act ? a + per : act;
  uint32_t s = 0;
  for (int64_t i = a; i < b; ++i) s += row[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 partials
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    uint32_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int64_t i = a; i < b; ++i) { uint32_t v = row[i]; row[i] = run; run += v; }
  if (threadIdx.x == blockDim.x - 1) rowtot[blockIdx.x] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_scatter(const uint64_t* __restrict__ key,
                                                          const uint32_t* __restrict__ idx,
                                                          const unsigned long long* __restrict__ n_dev, int64_t nblk,
                                                          int shift, const uint32_t* __restrict__ cnt,
                                                          const uint32_t* __restrict__ rowtot,
                                                          uint64_t* __restrict__ okey, uint32_t* __restrict__ oidx) {
  __shared__ uint32_t wc[kSortThreads / 32][256];
  __shared__ uint32_t dbase[256];
  const int64_t n = (int64_t)*n_dev;
  const int64_t act = (n + kSortTile - 1) / kSortTile;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // digit bases: exclusive scan of the row totals (thread d sums serially over 256 -> cheap)
  uint32_t rbase = 0;
  for (int d = 0; d < (int)threadIdx.x; ++d) rbase += rowtot[d];
  for (int64_t t = blockIdx.x; t < act; t += gridDim.x) {
    const int64_t base = t * kSortTile;
    for (int d = threadIdx.x; d < 256 * (kSortThreads / 32); d += kSortThreads) (&wc[0][0])[d] = 0;
    dbase[threadIdx.x] = rbase + cnt[(int64_t)threadIdx.x * nblk + t];
    __syncthreads();
    uint64_t kv[kSortItems];
    uint32_t iv[kSortItems];
    uint32_t rk[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      int64_t j = base + (int64_t)w * (32 * kSortItems) + i * 32 + lane;
      bool v = j < n;
      kv[i] = v ? key[j] : 0;
      iv[i] = v ? idx[j] : 0;
      unsigned d = v ? ((unsigned)(kv[i] >> shift) & 255u) : 256u;
      unsigned peers = __match_any_sync(0xffffffffu, d);
      unsigned b = d < 256u ? wc[w][d] : 0u;
      __syncwarp();
      if (d < 256u && lane == __ffs(peers) - 1) wc[w][d] = b + __popc(peers);
      __syncwarp();
      rk[i] = v ? (b + __popc(peers & lt)) | (d << 20) : 0xffffffffu;
    }
    __syncthreads();
    // exclusive scan over warps for each digit
    {
      uint32_t run = 0;
      for (int ww = 0; ww < kSortThreads / 32; ++ww) {
        uint32_t x = wc[ww][threadIdx.x];
        wc[ww][threadIdx.x] = run;
        run += x;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      if (rk[i] == 0xffffffffu) continue;
      unsigned d = rk[i] >> 20, r = rk[i] & 0xfffffu;
      uint32_t p = dbase[d] + wc[w][d] + r;
      okey[p] = kv[i];
      oidx[p] = iv[i];
    }
    __syncthreads();  // wc and dbase are rebuilt for the next tile
  }
}

void launch_radix_sort(uint64_t* key[2], uint32_t* idx[2], const unsigned long long* n_dev, int64_t n_max,
                       uint32_t* rcount, cudaStream_t s) {
  int64_t nblk = (n_max + kSortTile - 1) / kSortTile;
  if (nblk == 0) return;
  uint32_t* rowtot = rcount + 256 * nblk;
  // enough CTAs for about four per SM; they stride over the tiles the kept lines fill
  const unsigned grid = (unsigned)(nblk < 148 * 4 ? nblk : 148 * 4);
  for (int pass = 0; pass < 8; ++pass) {
    int src = pass & 1, dst = src ^ 1;
    int shift = pass * 8;
    k_hist<<<grid, kSortThreads, 0, s>>>(key[src], n_dev, nblk, shift, rcount);
    k_rowscan<<<256, 1024, 0, s>>>(rcount, n_dev, nblk, rowtot);
    k_scatter<<<grid, kSortThreads, 0, s>>>(key[src], idx[src], n_dev, nblk, shift, rcount, rowtot,
                                                      key[dst], idx[dst]);
  }
  note_launches(24);
}

// ------------------------------------------------------------------ list exponent
// k = frexp exponent of the largest kept |intensity| (R12); in accumulate mode the
// running sum's exponent is raised to max(k_run, k) and the sum rescaled exactly.
__global__ void k_exponent(const unsigned long long* maxbits, int32_t* kexp, int32_t* sig_exp, int accumulate) {
  double mx = __longlong_as_double((long long)*maxbits);
  int k = 0;
  if (mx > 0.0) frexp(mx, &k);
  if (accumulate && sig_exp) {
    int old = *sig_exp;
    if (old != PXC_EXP_EMPTY && (old > k || !(mx > 0.0))) k = old;
    kexp[1] = old;  // previous exponent, for the rescale kernel
  }
  kexp[0] = k;
  if (sig_exp) *sig_exp = k;
}

__global__ void k_rescale(float* sigma, int64_t n, const int32_t* kexp) {
  int old = kexp[1], k = kexp[0];
  if (old == PXC_EXP_EMPTY || old == k) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sigma[i] = ldexpf(sigma[i], old - k);
}

void launch_exponent(const unsigned long long* maxbits, int32_t* kexp, int32_t* sigma_exp_inout, int accumulate,
                     float* sigma, int64_t n_grid, cudaStream_t s) {
  k_exponent<<<1, 1, 0, s>>>(maxbits, kexp, sigma_exp_inout, accumulate);
  note_launches(1);
  if (accumulate && sigma) { k_rescale<<<592, 256, 0, s>>>(sigma, n_grid, kexp); note_launches(1); }
}

// ------------------------------------------------------------------ prepare sorted lines
// pos = {ic, f, ilo, ihi} with (nu - nu_min)/dnu = ic + f, par = {gamma_ref, n_T}, Is = ldexp(I, -k).
__global__ void __launch_bounds__(256) k_prepare(const uint64_t* __restrict__ skey, const uint32_t* __restrict__ sidx,
                                                 const unsigned long long* __restrict__ n_dev, GridP gp,
                                                 const float* __restrict__ gref, const float* __restrict__ nT,
                                                 const double* __restrict__ Iv, const int32_t* __restrict__ kexp,
                                                 int4* __restrict__ pos, float2* __restrict__ par,
                                                 float* __restrict__ Is, const int32_t* __restrict__ up,
                                                 const int32_t* __restrict__ lo, const void* __restrict__ Av, int A32,
                                                 int32_t* __restrict__ su, int32_t* __restrict__ sl,
                                                 double* __restrict__ sA, int64_t* __restrict__ perm,
                                                 unsigned long long* __restrict__ counters) {
  const int64_t n = (int64_t)*n_dev;
  const int k = Iv ? kexp[0] : 0;
  const double sk = pow2_scale(k);
  unsigned long long ev = 0, evnz = 0, nz = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double nu = key_nu(skey[j], gp);
    uint32_t t = sidx[j];
    int64_t a = 0, b = -1;
    exact_window(nu, gp, &a, &b);
    // position in grid steps: (nu - nu_min)/dnu, or (U/nu - lambda_min)/dlambda on a wavelength grid
    // (on a wavenumber grid by the reciprocal: the position only places the profile's centre, and
    // a last-bit difference moves it by ~1e-16 of its value; the window above is exact)
    double c = gp.wl_unit > 0.0 ? __ddiv_rn(__dsub_rn(__ddiv_rn(gp.wl_unit, nu), gp.nu_min), gp.dnu)
                                : __dsub_rn(nu, gp.nu_min) * gp.inv_dnu;
    double fc = floor(c);
    float f = (float)__dsub_rn(c, fc);
    pos[j] = make_int4((int)fc, __float_as_int(f), (int)a, (int)b);
    par[j] = (gref && nT) ? make_float2(gref[t], nT[t]) : make_float2(0.f, 0.f);
    unsigned long long wsz = (unsigned long long)(b - a + 1);
    ev += wsz;
    if (Iv) {
      float is = (float)scale_by(Iv[t], k, sk);
      Is[j] = is;
      if (is != 0.f) { evnz += wsz; ++nz; }
    }
    if (su && up) {
      su[j] = up[t];
      sl[j] = lo[t];
      sA[j] = A32 ? (double)((const float*)Av)[t] : ((const double*)Av)[t];
    }
    if (perm) perm[j] = (int64_t)t;
  }
  ev = warp_sum(ev); evnz = warp_sum(evnz); nz = warp_sum(nz);
  if ((threadIdx.x & 31) == 0) {
    if (ev) atomicAdd(&counters[CNT_EVALS], ev);
    if (evnz) atomicAdd(&counters[CNT_EVALS_NZ], evnz);
    if (nz) atomicAdd(&counters[CNT_NONZERO], nz);
  }
}

void launch_prepare(const uint64_t* skey, const uint32_t* sidx, const unsigned long long* n_dev, int64_t n_max,
                    const GridP& gp, const float* gamma_ref, const float* n_T, const double* Iv,
                    const int32_t* kexp, int4* pos, float2* par, float* Is,
                    const pxc_transitions* gather_tr, int32_t* su, int32_t* sl, double* sA,
                    int64_t* perm_out, unsigned long long* counters, cudaStream_t s) {
  if (n_max == 0) return;
  int64_t blocks = (n_max + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (!gather_tr) su = nullptr, sl = nullptr, sA = nullptr;  // no transition arrays: nothing to gather
  k_prepare<<<(unsigned)blocks, 256, 0, s>>>(skey, sidx, n_dev, gp, gamma_ref, n_T, Iv, kexp, pos, par, Is,
                                            gather_tr ? gather_tr->upper : nullptr,
                                            gather_tr ? gather_tr->lower : nullptr,
                                            gather_tr ? gather_tr->A : nullptr, gather_tr ? gather_tr->A_is_f32 : 0,
                                            su, sl, sA, perm_out, counters);
  note_launches(1);
}

// ------------------------------------------------------------------ batched intensities in sorted order
__global__ void __launch_bounds__(256) k_sorted_intensity(const int32_t* __restrict__ su, const int32_t* __restrict__ sl,
                                                          const double* __restrict__ sA,
                                                          const unsigned long long* __restrict__ n_dev,
                                                          const int32_t* __restrict__ g,
                                                          const double2* __restrict__ srec,
                                                          const double* __restrict__ qres, BoundP bp,
                                                          double threshold, double* __restrict__ sI,
                                                          unsigned long long* __restrict__ maxbits) {
  const int64_t n = (int64_t)*n_dev;
  const double invQ = qres[3];
  unsigned long long mx = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = su[j], l = sl[j];
    double2 ru = srec[u], rl = srec[l];
    double nu = __dsub_rn(ru.x, rl.x);
    double num, den;
    line_value(bp.mode, bp.c2_Td, (double)g[u], sA[j], invQ, rl.y, ru.y, nu, &num, &den);
    double I = fabs(num) >= threshold * den ? num / den : 0.0;
    sI[j] = I;
    unsigned long long ib = (unsigned long long)__double_as_longlong(fabs(I));
    mx = ib > mx ? ib : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long v = __shfl_down_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxbits, mx);
}

void launch_sorted_intensity(const int32_t* su, const int32_t* sl, const double* sA, const unsigned long long* n_dev,
                             int64_t n_max, const int32_t* g, const double2* srec, const double* qres,
                             const BoundP& bp, double threshold, double* sI, unsigned long long* maxbits,
                             cudaStream_t s) {
  if (n_max == 0) return;
  int64_t blocks = (n_max + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_sorted_intensity<<<(unsigned)blocks, 256, 0, s>>>(su, sl, sA, n_dev, g, srec, qres, bp, threshold, sI, maxbits);
  note_launches(1);
}

__global__ void k_scale(const double* __restrict__ sI, const unsigned long long* __restrict__ n_dev,
                        const int32_t* __restrict__ kexp, float* __restrict__ Is) {
  const int64_t n = (int64_t)*n_dev;
  const int k = kexp[0];
  const double sk = pow2_scale(k);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    Is[j] = (float)scale_by(sI[j], k, sk);
}

void launch_scale(const double* sI, const unsigned long long* n_dev, int64_t n_max, const int32_t* kexp,
                  float* Is, unsigned long long* counters, cudaStream_t s) {
  (void)counters;
  if (n_max == 0) return;
  int64_t blocks = (n_max + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_scale<<<(unsigned)blocks, 256, 0, s>>>(sI, n_dev, kexp, Is);
  note_launches(1);
}

// ------------------------------------------------------------------ segment binning
// Windows are monotone in nu, so the lines meeting segment s = [s S, (s+1) S) are the
// contiguous sorted range [first, last): first = #lines with ihi < s S, last = #lines with ilo <= (s+1) S - 1.
__global__ void k_segments(const int4* __restrict__ pos, const unsigned long long* __restrict__ n_dev, int64_t nseg,
                           int seg, int32_t* __restrict__ segr) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int64_t n = (int64_t)*n_dev;
  const int64_t a = s * seg, b = (s + 1) * seg - 1;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if ((int64_t)pos[m].w < a) lo = m + 1; else hi = m;
  }
  int64_t first = lo;
  lo = first; hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if ((int64_t)pos[m].z <= b) lo = m + 1; else hi = m;
  }
  segr[s] = (int32_t)first;
  segr[nseg + s] = (int32_t)lo;
}

void launch_segments(const int4* pos, const unsigned long long* n_dev, int64_t nseg, int seg, int32_t* segr,
                     cudaStream_t s) {
  k_segments<<<(unsigned)((nseg + 255) / 256), 256, 0, s>>>(pos, n_dev, nseg, seg, segr);
  note_launches(1);
}

// Work items: each (condition, segment) group is split into ceil(lines / item_lines) items (at least one).
// Work items of the profile kernel, in four launches over all (condition, segment) pairs:
// total line-segment pairs (integer atomics), items per pair, exclusive scan, emission.
// Lines per item: about target_items equal items over all segments (load balance of the
// persistent profile kernel), at least 512, never more split items than partial rows; only
// the single-condition call splits (its partial rows are reduced), batched calls use
// item_lines_max.
__device__ __forceinline__ int item_lines_of(unsigned long long all, int item_lines_max, int64_t target_items,
                                             int64_t max_partial) {
  long long L = item_lines_max;
  if (target_items > 0) {
    long long t = (long long)((all + target_items - 1) / target_items);
    long long m = (long long)((all + max_partial - 1) / (max_partial > 0 ? max_partial : 1));
    t = t > 512 ? t : 512;
    t = t > m ? t : m;
    t = (t + 255) / 256 * 256;
    L = t < item_lines_max ? t : item_lines_max;
  }
  return (int)L;
}

__global__ void __launch_bounds__(256) k_items_total(const int32_t* __restrict__ segr, int64_t nseg,
                                                     unsigned long long* __restrict__ counters) {
  unsigned long long tot = 0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x)
    tot += (unsigned long long)(segr[nseg + s] - segr[s]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&counters[CNT_ALL], tot);
}

__global__ void __launch_bounds__(256) k_items_count(const int32_t* __restrict__ segr, int64_t nseg, int n_c,
                                                     int item_lines_max, const unsigned long long* __restrict__ counters,
                                                     int64_t target_items, int64_t max_partial,
                                                     uint32_t* __restrict__ cnt) {
  const int L = item_lines_of(counters[CNT_ALL] * (unsigned long long)n_c, item_lines_max, target_items, max_partial);
  const int64_t ng = nseg * n_c;
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < ng; gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = gi % nseg;
    const int64_t nl = (int64_t)segr[nseg + s] - segr[s];
    const int64_t c = (nl + L - 1) / L;
    cnt[gi] = (uint32_t)(c < 1 ? 1 : c);
  }
}

__global__ void __launch_bounds__(256) k_items_emit(const int32_t* __restrict__ segr, int64_t nseg, int n_c,
                                                    int item_lines_max, const int32_t* __restrict__ seg_items,
                                                    Item* __restrict__ items, unsigned long long* __restrict__ counters,
                                                    int64_t max_items, int64_t target_items, int64_t max_partial,
                                                    const int32_t* __restrict__ cond_list) {
  const int L = item_lines_of(counters[CNT_ALL] * (unsigned long long)n_c, item_lines_max, target_items, max_partial);
  const int64_t ng = nseg * n_c;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long run = (unsigned long long)(uint32_t)seg_items[ng];
    counters[CNT_ITEMS] = run < (unsigned long long)max_items ? run : (unsigned long long)max_items;
    counters[CNT_QUEUE] = 0;
  }
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < ng; gi += (int64_t)gridDim.x * blockDim.x) {
    const int32_t first = seg_items[gi], c = seg_items[gi + 1] - first;
    const int64_t s = gi % nseg;
    const int32_t f = segr[s], e = segr[nseg + s];
    for (int32_t k = 0; k < c; ++k) {
      const int64_t idx = (int64_t)first + k;
      if (idx >= max_items) break;  // sized on the host; never taken for calls that passed the capacity check
      Item it;
      it.cond = cond_list ? cond_list[gi / nseg] : (int32_t)(gi / nseg);
      it.seg = (int32_t)s;
      it.begin = (int32_t)(f + (int64_t)k * L);
      const int64_t en = (int64_t)f + (int64_t)(k + 1) * L;
      it.end = (int32_t)(en < e ? en : e);
      if (it.begin > e) it.begin = e;
      it.slot = k == 0 ? -1 : (int32_t)(idx - gi - 1);
      it.first_of_seg = first;
      it.n_of_seg = c;
      it.pad = 0;
      items[idx] = it;
    }
  }
}

void launch_items(const int32_t* segr, int64_t nseg, int n_c, int item_lines, int32_t* seg_items, Item* items,
                  unsigned long long* counters, int64_t max_items, int64_t target_items, int64_t max_partial,
                  const int32_t* cond_list, cudaStream_t s) {
  const int64_t ng = nseg * n_c;
  cudaMemsetAsync(counters + CNT_ALL, 0, sizeof(unsigned long long), s);
  auto blocks = [](int64_t n) { int64_t b = (n + 255) / 256; return (unsigned)(b < 1 ? 1 : (b > 148 * 8 ? 148 * 8 : b)); };
  k_items_total<<<blocks(nseg), 256, 0, s>>>(segr, nseg, counters);
  k_items_count<<<blocks(ng), 256, 0, s>>>(segr, nseg, n_c, item_lines, counters, target_items, max_partial,
                                           reinterpret_cast<uint32_t*>(seg_items));
  k_scan_counts<<<1, 1024, 0, s>>>(reinterpret_cast<uint32_t*>(seg_items), ng, counters + CNT_ITEMS_RAW);
  k_items_emit<<<blocks(ng), 256, 0, s>>>(segr, nseg, n_c, item_lines, seg_items, items, counters, max_items,
                                          target_items, max_partial, cond_list);
  note_launches(4);
}

// Adds the partial rows of split segments to sigma, in item order (deterministic).
__global__ void k_reduce_partials(const Item* __restrict__ items, const int32_t* __restrict__ seg_items, int64_t nseg,
                                  int seg, const float* __restrict__ partial, float* __restrict__ sigma,
                                  int64_t n_grid, const int32_t* __restrict__ cond_list) {
  int64_t gi = blockIdx.x;
  int32_t f = seg_items[gi], e = seg_items[gi + 1];
  if (e - f <= 1) return;
  const int64_t s = gi % nseg, c = cond_list ? cond_list[gi / nseg] : gi / nseg;
  for (int p = threadIdx.x; p < seg; p += blockDim.x) {
    int64_t i = s * seg + p;
    if (i >= n_grid) break;
    float v = sigma[c * n_grid + i];
    for (int32_t it = f + 1; it < e; ++it) v += partial[(int64_t)items[it].slot * seg + p];
    sigma[c * n_grid + i] = v;
  }
}

void launch_reduce_partials(const Item* items, const int32_t* seg_items, int64_t nseg, int seg, int n_c,
                            const float* partial, float* sigma, int64_t n_grid, const int32_t* cond_list,
                            cudaStream_t s) {
  k_reduce_partials<<<(unsigned)(nseg * n_c), 128, 0, s>>>(items, seg_items, nseg, seg, partial, sigma, n_grid,
                                                           cond_list);
  note_launches(1);
}

// ------------------------------------------------------------------ stick-spectrum output
__global__ void k_stick_out(const double* __restrict__ Iv, const uint64_t* __restrict__ key, int64_t n,
                            const int32_t* __restrict__ kexp, float* __restrict__ out) {
  const int k = kexp[0];
  const double sk = pow2_scale(k);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = key[t] == kSentinelKey ? 0.f : (float)scale_by(Iv[t], k, sk);
}

void launch_stick_out(const double* Iv, const uint64_t* key, int64_t n, const int32_t* kexp, float* I_scaled,
                      cudaStream_t s) {
  if (n == 0) return;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  k_stick_out<<<(unsigned)blocks, 256, 0, s>>>(Iv, key, n, kexp, I_scaled);
  note_launches(1);
}

}  // namespace pxc
