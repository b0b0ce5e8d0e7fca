// Profile accumulation (Eq. xsec over the kept lines) and its adjoint.
//
// Forward: persistent CTAs take work items (condition, grid segment of S points,
// a contiguous range of the nu-sorted lines whose windows meet the segment);
// S and the CTA shape are one of the compiled tile configurations.  Each lane
// owns points of the segment in registers.  The line records (position,
// broadening parameters, scaled intensity) are staged into shared memory by
// 1-D bulk TMA copies (cp.async.bulk) completing on mbarriers; every wait is
// bounded.  Each warp turns the staged records into its own line constants and
// classes and evaluates its lines at its points in FP32, with no atomics; stage
// sums are added into per-item sums (two-level summation).
//
// Voigt uses Humlicek's W4 rational approximation of the Faddeeva function
// (J. Humlicek, JQSRT 27 (1982) 437), the method the paper recommends for GPU
// Voigt evaluation (Sec. 4.1): region I (|x|+y >= 15) is the one-level
// Laplace continued fraction t/sqrt(pi)/(1/2 + t^2), t = y - ix, whose real part
// needs one reciprocal; lines whose whole segment lies in region I and inside
// the cut-off window take a branch-free path.
#include <cstdio>

#include "kernels.cuh"

namespace pxc {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Bounded wait: true if the phase completed, false after `limit` clock cycles.
// Non-blocking probe of a phase (try_wait may suspend the thread for a while before failing).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for a phase for at most `limit` clock cycles; a limit of 0 only probes it once.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
  if (limit == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ float frcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ------------------------------------------------------------------ Humlicek W4 (FP32)
struct cplx {
  float r, i;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cplx cadd(cplx a, float b) { return {a.r + b, a.i}; }
__device__ __forceinline__ cplx csub_from(float a, cplx b) { return {a - b.r, -b.i}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  float d = frcp(b.r * b.r + b.i * b.i);
  return {(a.r * b.r + a.i * b.i) * d, (a.i * b.r - a.r * b.i) * d};
}

// Complex W4 value w(z) and dw/dz, z = x + iy (y >= 0).  Regions as published:
// I: s >= 15, II: 5.5 <= s < 15, III: s < 5.5 and y >= 0.195|x| - 0.176, IV otherwise.
__device__ __noinline__ void w4_full(float x, float y, cplx* w, cplx* dw) {
  const float ax = fabsf(x), s = ax + y;
  const cplx t = {y, -x};
  const cplx u = cmul(t, t);
  cplx dwdt;
  if (s >= 15.f) {
    // w = t N / D, N = 1/sqrt(pi), D = 1/2 + u;  dw/dt = N (1/2 - u) / D^2
    cplx D = cadd(u, 0.5f);
    *w = cdiv({t.r * kInvSqrtPi, t.i * kInvSqrtPi}, D);
    cplx D2 = cmul(D, D);
    dwdt = cdiv({kInvSqrtPi * (0.5f - u.r), -kInvSqrtPi * u.i}, D2);
  } else if (s >= 5.5f) {
    // w = t N(u) / D(u), N = a + b u, D = c + 3u + u^2; dw/dt = [N D + 2u (N' D - N D')] / D^2
    const float a = 1.410474f, b = 0.5641896f;
    cplx N = {a + b * u.r, b * u.i};
    cplx D = cadd(cmul(u, cadd(u, 3.f)), 0.75f);
    *w = cdiv(cmul(t, N), D);
    cplx Dp = {3.f + 2.f * u.r, 2.f * u.i};
    cplx inner = {b * D.r - (N.r * Dp.r - N.i * Dp.i), b * D.i - (N.r * Dp.i + N.i * Dp.r)};
    cplx two_u = {2.f * u.r, 2.f * u.i};
    cplx num = cmul(N, D);
    cplx add = cmul(two_u, inner);
    dwdt = cdiv({num.r + add.r, num.i + add.i}, cmul(D, D));
  } else if (y >= 0.195f * ax - 0.176f) {
    // w = P(t) / Q(t)
    cplx P = cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, {0.5642236f, 0.f}), 3.778987f)), 11.96482f)), 20.20933f)),
                  16.4955f);
    cplx Q = cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd(t, 6.699398f)), 21.69274f)), 39.27121f)),
                               38.82363f)),
                  16.4955f);
    *w = cdiv(P, Q);
    // derivatives of the polynomials
    cplx Pp = cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, {4.f * 0.5642236f, 0.f}), 3.f * 3.778987f)), 2.f * 11.96482f)),
                   20.20933f);
    cplx Qp = cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd({5.f * t.r, 5.f * t.i}, 4.f * 6.699398f)), 3.f * 21.69274f)),
                               2.f * 39.27121f)),
                   38.82363f);
    cplx a1 = cmul(Pp, Q), a2 = cmul(P, Qp);
    dwdt = cdiv({a1.r - a2.r, a1.i - a2.i}, cmul(Q, Q));
  } else {
    // w = exp(u) - t P(u) / Q(u)
    cplx P = csub_from(36183.31f, cmul(u, csub_from(3321.9905f, cmul(u, csub_from(1540.787f, cmul(u, csub_from(219.0313f,
                 cmul(u, csub_from(35.76683f, cmul(u, csub_from(1.320522f, {0.56419f * u.r, 0.56419f * u.i})))))))))));
    cplx Q = csub_from(32066.6f, cmul(u, csub_from(24322.84f, cmul(u, csub_from(9022.228f, cmul(u, csub_from(2186.181f,
                 cmul(u, csub_from(364.2191f, cmul(u, csub_from(61.57037f, cmul(u, csub_from(1.841439f, u)))))))))))));
    float eu = expf(u.r);
    float sn, cs;
    sincosf(u.i, &sn, &cs);
    cplx e = {eu * cs, eu * sn};
    cplx R = cdiv(P, Q);
    cplx tR = cmul(t, R);
    *w = {e.r - tR.r, e.i - tR.i};
    // P'(u), Q'(u)
    cplx Pp = {-3321.9905f, 0.f};
    {
      // P(u) = 36183.31 - 3321.9905 u + 1540.787 u^2 - 219.0313 u^3 + 35.76683 u^4 - 1.320522 u^5 + 0.56419 u^6
      const float c[7] = {36183.31f, -3321.9905f, 1540.787f, -219.0313f, 35.76683f, -1.320522f, 0.56419f};
      cplx acc = {6.f * c[6], 0.f};
      for (int k = 5; k >= 1; --k) acc = cadd(cmul(acc, u), (float)k * c[k]);
      Pp = acc;
    }
    cplx Qp;
    {
      // Q(u) = 32066.6 - 24322.84 u + 9022.228 u^2 - 2186.181 u^3 + 364.2191 u^4 - 61.57037 u^5 + 1.841439 u^6 - u^7
      const float c[8] = {32066.6f, -24322.84f, 9022.228f, -2186.181f, 364.2191f, -61.57037f, 1.841439f, -1.f};
      cplx acc = {7.f * c[7], 0.f};
      for (int k = 6; k >= 1; --k) acc = cadd(cmul(acc, u), (float)k * c[k]);
      Qp = acc;
    }
    // d/dt [t R(u)] = R + 2u R'(u), R' = (P'Q - PQ')/Q^2
    cplx a1 = cmul(Pp, Q), a2 = cmul(P, Qp);
    cplx Rp = cdiv({a1.r - a2.r, a1.i - a2.i}, cmul(Q, Q));
    cplx two_u = {2.f * u.r, 2.f * u.i};
    cplx dtR = cmul(two_u, Rp);
    cplx two_t_e = cmul({2.f * t.r, 2.f * t.i}, e);
    dwdt = {two_t_e.r - R.r - dtR.r, two_t_e.i - R.i - dtR.i};
  }
  // t = -i z  =>  dw/dz = -i dw/dt
  *dw = {dwdt.i, -dwdt.r};
}

// Real part of W4 in regions II-IV (|x| + y < 15), forward only.  Kept out of line so the
// branch-free far-wing loop of the profile kernel stays small in registers.
// W4 region III (|x|+y < 5.5, y >= 0.195|x| - 0.176): a degree-5 rational in t = y - ix.
__device__ __forceinline__ float w4_reg3_re(float x, float y) {
  const cplx t = {y, -x};
  cplx P = cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, {0.5642236f, 0.f}), 3.778987f)), 11.96482f)), 20.20933f)),
                16.4955f);
  cplx Q = cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd(cmul(t, cadd(t, 6.699398f)), 21.69274f)), 39.27121f)),
                             38.82363f)),
                16.4955f);
  return cdiv(P, Q).r;
}

// W4 region IV (the rest of |x|+y < 5.5): w = exp(u) - t P(u)/Q(u), u = t^2.  The hardware
// exp2/cos approximations cost ~1e-6 absolute in e^Re(u) cos(Im u) for |Im u| <= 11 here,
// two orders below the W4 accuracy.
__device__ __forceinline__ float w4_reg4_re(float x, float y) {
  const cplx t = {y, -x};
  const cplx u = cmul(t, t);
  cplx P = csub_from(36183.31f, cmul(u, csub_from(3321.9905f, cmul(u, csub_from(1540.787f, cmul(u, csub_from(219.0313f,
               cmul(u, csub_from(35.76683f, cmul(u, csub_from(1.320522f, {0.56419f * u.r, 0.56419f * u.i})))))))))));
  cplx Q = csub_from(32066.6f, cmul(u, csub_from(24322.84f, cmul(u, csub_from(9022.228f, cmul(u, csub_from(2186.181f,
               cmul(u, csub_from(364.2191f, cmul(u, csub_from(61.57037f, cmul(u, csub_from(1.841439f, u)))))))))))));
  return __expf(u.r) * __cosf(u.i) - cmul(t, cdiv(P, Q)).r;
}

__device__ __noinline__ float w4_core_re(float x, float y) {
  const float ax = fabsf(x), s = ax + y;
  if (s >= 5.5f) {
    // w = t (1.410474 + 0.5641896 u) / (0.75 + u (3 + u))
    const cplx t = {y, -x};
    const cplx u = cmul(t, t);
    cplx N = {1.410474f + 0.5641896f * u.r, 0.5641896f * u.i};
    cplx D = cadd(cmul(u, cadd(u, 3.f)), 0.75f);
    return cdiv(cmul(t, N), D).r;
  }
  if (y >= 0.195f * ax - 0.176f) return w4_reg3_re(x, y);
  return w4_reg4_re(x, y);
}

// Region-I (far-wing) Voigt term K (u + 1) / (u^2 + e), u = x^2 + y^2 - 1/2, in the form
// K (1 + 1/u) / (u + e/u), which stays finite for any representable u (u^2 would overflow FP32
// beyond |x| ~ 4e9); u >= 200 wherever region I applies.  The fast path uses the direct form on
// constants rescaled per warp instead (scale_for_pairs).
__device__ __forceinline__ float region_one(float u, float K, float e) {
  const float r = frcp(u);
  return K * (1.f + r) * frcp(fmaf(e, r, u));
}
// LineC::masks bit set when a line's region-I terms in a warp need region_one (|x| or y >= 1e9);
// otherwise the direct K (u + 1) / (u^2 + e), one reciprocal, is used.
constexpr int kWideRange = 8;
// LineC::masks bit set when every |x| of a line in a warp is below 1e4: region II's quartic in
// x^2 then stays far inside the FP32 range, and the core and mid paths use it for every point
// with |x| + y >= 5.5 (it is at least as accurate as region I there), one path fewer.
constexpr int kRegion2Everywhere = 16;
__device__ __forceinline__ float region_one_or_direct(float u, float K, float e, int masks) {
  return (masks & kWideRange) ? region_one(u, K, e) : fmaf(u, K, K) * frcp(fmaf(u, u, e));
}

// Real part of W4 in every region (used by the general path).
__device__ __forceinline__ float w4_re(float x, float y) {
  const float ax = fabsf(x), s = ax + y;
  if (s >= 15.f) return region_one(fmaf(x, x, fmaf(y, y, -0.5f)), kInvSqrtPi * y, 2.f * y * y);
  return w4_core_re(x, y);
}

// ------------------------------------------------------------------ forward kernel
// A CTA of THREADS threads takes work items on a segment of SEG = THREADS * PTS grid
// points.  Warp w owns the points [32 PTS w, 32 PTS (w + 1)); lane l holds the points
// 32 PTS w + l + 32 k, k < PTS, in registers.  The segment width and the lines per stage
// are template parameters: the tile configurations below are compiled, and the workspace
// picks one per profile kind (pxc_autotune times them on the caller's inputs).

struct __align__(16) LineC {
  // fast-path constants, first so that two 16-byte loads fetch them:
  //   Voigt:   a = x at lane 0 of the owning warp, b = step, B1 = c1 = y^2 - 1/2, d = e = 2 y^2
  //   others:  a = wbase - pf (exact integer), b = step, B1 = gamma^2 (Lorentz) or 0, d = nfs
  float a, b, B1, d;
  float K, KA, y, Kc;          // amplitudes (K: fast/region I, Kc: general path), y (Voigt) or gamma
  float pf, step, nfs, reach;  // centre offset (grid steps, exact integer part), step, -f*step;
                               // half-width of the non-region-I zone (grid steps)
  int lo, hi;                  // window relative to the segment (grid points, clamped)
  int masks;                   // 1 if the line is valid with non-zero intensity and a non-empty window; then its class
  float cen;                   // the centre (grid steps from the segment start)
};

// Smallest Doppler HWHM used by the sampled Gaussian and Voigt kinds (cm^-1): 1/alpha^2 stays a
// normal FP32 number (the far-wing terms away from the fast path use the overflow-free form of
// region_one above, so a grid step of up to ~1e13 Doppler widths is fine).  Only lines with nu below
// ~3e-10 cm^-1 are floored.
constexpr float kAlphaMin = 1e-15f;
// The floor of the binned and pseudo-Voigt kinds and of the adjoint, whose bin-mass, common-width
// and derivative arithmetic is kept finite by it: lines with nu below ~0.05 cm^-1, whose true
// alpha is far below both the grid step and gamma (the sampled profile changes by less than
// (alpha/gamma)^2 off the line centre).
constexpr float kAlphaMinWide = 8.4e-8f;

// Smallest Lorentz HWHM used (cm^-1): gamma^2 stays a normal FP32 number.
constexpr float kGammaMin = 1e-15f;

// Pseudo-Voigt profiles (Table profile: Thompson, Olivero, Liu-Lin): a Lorentzian and a Gaussian
// of one common full width G, weights wL and wG, from the Doppler and Lorentz HWHMs alpha, gamma
// (full widths fG = 2 alpha, fL = 2 gamma):
//   Thompson (Thompson, Cox, Hastings 1987): G^5 = fG^5 + 2.69269 fG^4 fL + 2.42843 fG^3 fL^2
//     + 4.47163 fG^2 fL^3 + 0.07842 fG fL^4 + fL^5, wL = 1.36603 r - 0.47719 r^2 + 0.11116 r^3,
//     r = fL / G, wG = 1 - wL (the fifth power is taken of the widths over the larger one, so no
//     FP32 over- or underflow);
//   Olivero (Olivero, Longbothum 1977): G = 0.5346 fL + sqrt(0.2166 fL^2 + fG^2), the same mixing;
//   Liu-Lin (Liu, Lin et al. 2001): d = (fL - fG)/(fL + fG), G = (fL + fG)(1 - 0.18121 (1 - d^2)
//     - (0.023665 e^{0.6 d} + 0.00418 e^{-1.9 d}) sin(pi d)), wL = 0.68188 + 0.61293 d - 0.18384 d^2
//     - 0.11568 d^3, wG = 0.32460 - 0.61825 d + 0.17681 d^2 + 0.12109 d^3.
template <int KIND>
__device__ __forceinline__ void pv_params(float alpha, float gamma, float* G, float* wl, float* wg) {
  const float fG = 2.f * alpha, fL = 2.f * gamma;
  if (KIND == PXC_PV_LIULIN) {
    const float d = (fL - fG) * frcp(fL + fG);
    *G = (fL + fG) * (1.f - 0.18121f * fmaf(-d, d, 1.f) -
                      (0.023665f * __expf(0.6f * d) + 0.00418f * __expf(-1.9f * d)) * sinpif(d));
    *wl = fmaf(fmaf(fmaf(-0.11568f, d, -0.18384f), d, 0.61293f), d, 0.68188f);
    *wg = fmaf(fmaf(fmaf(0.12109f, d, 0.17681f), d, -0.61825f), d, 0.32460f);
    return;
  }
  if (KIND == PXC_PV_THOMPSON) {
    const float u = fmaxf(fG, fL), iu = frcp(u);
    const float g = fG * iu, l = fL * iu;
    const float g2 = g * g, l2 = l * l;
    const float s5 = g2 * g2 * g + 2.69269f * g2 * g2 * l + 2.42843f * g2 * g * l2 + 4.47163f * g2 * l2 * l +
                     0.07842f * g * l2 * l2 + l2 * l2 * l;
    *G = u * exp2f(0.2f * __log2f(s5));
  } else {
    *G = fmaf(0.5346f, fL, sqrtf(fmaf(0.2166f * fL, fL, fG * fG)));
  }
  const float r = fL * frcp(*G);
  *wl = r * fmaf(fmaf(0.11116f, r, -0.47719f), r, 1.36603f);
  *wg = 1.f - *wl;
}

// Per-line constants for the warp owning points [wbase, wbase + 32 PTS) of the segment.  All
// FP32: the centre wavenumber that scales the Doppler width is rebuilt from the grid index and
// fraction (relative error ~1e-7, far below the profile tolerance); reciprocals are the
// hardware approximation (<= 1 ulp), and the region-I reach is widened by 1e-4 to stay safe.
template <int KIND, int SEG>
__device__ __forceinline__ void line_constants(const int4 p4, const float2 pr, const float is, const CondDev& cd,
                                               int64_t i0, int wbase, float dnu_f, float nu_min_f, bool valid,
                                               LineC& c) {
  const int ic = p4.x;
  const float f = __int_as_float(p4.y);
  // grid indices fit in 32 bits (the host caps the grid below 2^31 - 2 segments), so the
  // segment offsets are 32-bit integer arithmetic (a 64-bit conversion would use the FP64 pipe)
  const int i0i = (int)i0;
  c.pf = (float)(ic - i0i);
  const int lo = p4.z - i0i, hi = p4.w - i0i;
  c.lo = lo < 0 ? 0 : lo;
  c.hi = hi > SEG - 1 ? SEG - 1 : hi;
  const float cen = c.pf + f;  // line centre in grid steps from the segment start
  float reach = 0.f;           // half-width (grid steps) of the zone needing the general path
  if (is_binned(KIND)) {
    // Binned profiles: t = bin-centre offset in the kind's scaled unit; the bin is [t - h, t + h]
    // with h = step / 2 (see eval_binned).
    constexpr int BASE = KIND & 3;
    if (BASE == PXC_LORENTZ) {
      const float g = fmaxf(pr.x * exp2f(pr.y * cd.log2_tratio) * cd.P_f, kGammaMin);
      c.step = dnu_f * frcp(g);                // t in units of gamma
      c.B1 = fmaf(-0.25f * c.step, c.step, 1.f);  // 1 - h^2
      c.K = is * kInvPi * frcp(dnu_f);
      c.y = g;
    } else {
      const float nu = fmaf((float)ic + f, dnu_f, nu_min_f);
      const float alpha = fmaxf(BASE == PXC_GAUSS_HWHM ? cd.hwhm : cd.alpha_coef * nu, kAlphaMinWide);
      const float cc = kSqrtLn2 * frcp(alpha);  // 1 / (s sqrt 2)
      c.step = dnu_f * cc;
      if (BASE == PXC_VOIGT) {
        const float g = pr.x * exp2f(pr.y * cd.log2_tratio) * cd.P_f;
        c.y = g * cc;
        c.K = is * cc * kInvSqrtPi;
        c.d = fmaxf(kSqrtLn2, c.y);  // the larger width (alpha is sqrt(ln2) in this unit)
      } else {
        c.B1 = 0.5f * c.step;                   // h
        c.K = 0.5f * is * frcp(dnu_f);
        // provably-zero trim: erfcf(10.5) is below the FP32 range, so bins whose nearer edge
        // is beyond 10.5 carry no mass
        const float r = 10.5f * frcp(c.step) + 0.5f;
        const float elo = ceilf(cen - r), ehi = floorf(cen + r);
        if (elo > (float)c.lo) c.lo = (int)fminf(elo, (float)SEG);
        if (ehi < (float)c.hi) c.hi = (int)fmaxf(ehi, -1.f);
      }
    }
    c.nfs = -f * c.step;
    c.Kc = c.K;
    c.reach = 0.f;
    c.cen = cen;
    c.masks = (valid && is != 0.f && c.lo <= c.hi) ? 1 : 0;
    return;
  }
  if (is_pseudo_voigt(KIND)) {
    // t = (nu_i - nu_l) / h, h = G / 2: f = wL / (pi h (1 + t^2)) + wG sqrt(ln2 / pi) / h 2^(-t^2)
    const float nu = fmaf((float)ic + f, dnu_f, nu_min_f);
    const float alpha = fmaxf(cd.alpha_coef * nu, kAlphaMinWide);
    const float g = pr.x * exp2f(pr.y * cd.log2_tratio) * cd.P_f;
    float G, wl, wg;
    pv_params<KIND>(alpha, g, &G, &wl, &wg);
    const float ih = 2.f * frcp(G);
    c.step = dnu_f * ih;
    c.nfs = -f * c.step;
    c.K = is * wl * kInvPi * ih;
    c.KA = is * wg * (kSqrtLn2 * kInvSqrtPi) * ih;
    c.Kc = c.K;
    c.B1 = 0.f; c.y = 0.f;
    c.a = (float)wbase - c.pf;
    c.b = c.step;
    c.d = c.nfs;
  } else if (KIND == PXC_LORENTZ) {
    const float g = fmaxf(pr.x * exp2f(pr.y * cd.log2_tratio) * cd.P_f, kGammaMin);
    c.step = dnu_f;
    c.nfs = -f * dnu_f;
    c.B1 = g * g;
    c.Kc = is * g * kInvPi;
    c.K = c.Kc;
    c.KA = 0.f; c.y = g;
    c.a = (float)wbase - c.pf;
    c.b = c.step;
    c.d = c.nfs;
  } else {
    const float nu = fmaf((float)ic + f, dnu_f, nu_min_f);
    const float alpha = fmaxf(KIND == PXC_GAUSS_HWHM ? cd.hwhm : cd.alpha_coef * nu, kAlphaMin);
    const float cc = kSqrtLn2 * frcp(alpha);  // 1 / (s sqrt 2)
    if (KIND == PXC_VOIGT) {
      const float g = pr.x * exp2f(pr.y * cd.log2_tratio) * cd.P_f;
      const float y = g * cc;
      c.y = y;
      c.step = dnu_f * cc;
      c.nfs = -f * c.step;
      // region I: Re w = y (A + x^2) / (sqrt(pi) ((A - x^2)^2 + 4 x^2 y^2)), A = 1/2 + y^2, written
      // with v = x^2 + c1, c1 = y^2 - 1/2, as y (v + 1) / (sqrt(pi) (v^2 + e)), e = 2 y^2
      // (the denominator is the same quartic: (x^2 + c1)^2 + 2 y^2 = x^4 + (2y^2 - 1) x^2 + A^2)
      c.B1 = fmaf(y, y, -0.5f);
      c.d = 2.f * y * y;
      c.Kc = is * cc * kInvSqrtPi;
      c.K = c.Kc * y * kInvSqrtPi;
      c.KA = c.K;
      reach = fmaxf(15.f - y, 0.f) * frcp(c.step) * 1.0001f;
      c.a = fmaf((float)wbase - c.pf, c.step, c.nfs);
      c.b = c.step;
    } else {
      // exp(-X^2) = 2^(-(X sqrt(log2 e))^2); x is scaled by sqrt(log2 e)
      const float sl2e = 1.2011224087864498f;
      c.step = dnu_f * cc * sl2e;
      c.nfs = -f * c.step;
      c.Kc = is * cc * kInvSqrtPi;
      c.K = c.Kc;
      c.y = 0.f; c.B1 = 0.f; c.KA = 0.f;
      c.a = (float)wbase - c.pf;
      c.b = c.step;
      c.d = c.nfs;
      // provably-zero trim: ex2.approx.ftz flushes 2^(-t) to 0 for t > 126, and |X'| >= 12.7
      // (rounded reciprocal included) gives t >= 161
      const float r = 12.7f * frcp(c.step);
      const float elo = ceilf(cen - r), ehi = floorf(cen + r);
      if (elo > (float)c.lo) c.lo = (int)fminf(elo, (float)SEG);
      if (ehi < (float)c.hi) c.hi = (int)fmaxf(ehi, -1.f);
    }
  }
  c.reach = reach;
  c.cen = cen;
  c.masks = (valid && is != 0.f && c.lo <= c.hi) ? 1 : 0;
}

// Class of a line for the warp owning points [a, a + WPTS) of the segment:
// 0 nothing, 1 fast (inside the window, region I), 2 window edge (region I, lane mask),
// 3 near the line core (some point in W4 regions III/IV), 4 near the core but every point in
// regions I/II (Voigt only).
template <int KIND, int WPTS>
__device__ __forceinline__ int line_class(const LineC& c, int a) {
  const int b = a + WPTS - 1;
  if (!c.masks || c.hi < a || c.lo > b) return 0;
  if (is_binned(KIND)) return 2;  // binned kinds: one masked path (eval_binned)
  bool far = true;
  if (KIND == PXC_VOIGT) {
    const float dmin = fmaxf(0.f, fmaxf(c.cen - (float)b, (float)a - c.cen));
    far = dmin > c.reach;
  }
  if (!far) {
    // near the centre: 4 if every point still has |x| + y >= 5.5 (W4 region II or I), else 3
    const float dmin = fmaxf(0.f, fmaxf(c.cen - (float)b, (float)a - c.cen));
    const float reach5 = fmaxf(5.5f - c.y, 0.f) * frcp(c.step) * 1.0001f;
    return dmin > reach5 ? 4 : 3;
  }
  return (c.lo <= a && c.hi >= b) ? 1 : 2;
}


// Far-wing Voigt lines evaluated in pairs share one reciprocal: n1/d1 + n2/d2 = (n1 d2 + n2 d1) /
// (d1 d2).  To keep d1 d2 inside the FP32 range, each fast line's constants are rescaled for its
// warp by sigma = 2^-e, e the exponent of x_ref = max(min |x| over the warp's points, y): with
// x' = sigma x every term of K (v + 1) / (v^2 + e) scales exactly (v' = sigma^2 v, the numerator by
// sigma^2, the denominator by sigma^4), so the value is unchanged and the scaled denominators lie
// in [~1, 2^52] when max |x| <= 2^12 x_ref.  Returns false (the line then takes the masked
// single-line path) when the warp spans a wider range of |x| than that.
//
// Where |z|^2 = x^2 + y^2 >= kLorentzR2 at every point of the warp, the line's far wing is taken in
// its Lorentzian limit K / (x^2 + y^2) instead: the region-I value is
//   K (u + 1) / (u^2 + e) = (K / |z|^2) (|z|^4 + |z|^2 / 2) / (|z|^4 - x^2 + y^2 + 1/4)
//                         = (K / |z|^2) (1 + (3 x^2 - y^2) / (2 |z|^4) + O(|z|^-4)),
// so the limit is within 1.5 / |z|^2 <= 3e-5 of it (relative).  Such a line is marked by d < 0 and
// carries B1 = sigma^2 y^2 (its scaled denominator is x'^2 + B1); the staging keeps it as the
// float4 {a, b, B1, K}.  Two of them cost eight FP32 instructions and one reciprocal per point,
// against twelve and one for two region-I lines.
#ifndef PXC_LORENTZ_R2
#define PXC_LORENTZ_R2 5e4f
#endif
constexpr float kLorentzR2 = PXC_LORENTZ_R2;

template <int WPTS>
__device__ __forceinline__ bool scale_for_pairs(LineC& c, int wbase) {
  const float wlo = (float)wbase, whi = (float)(wbase + WPTS - 1);
  const float dmin = fmaxf(0.f, fmaxf(c.cen - whi, wlo - c.cen));
  const float dmax = fmaxf(fabsf(c.cen - wlo), fabsf(c.cen - whi));
  const float xm = dmin * c.step;
  const float xref = fmaxf(xm, c.y);
  if (!(xref > 0.f) || !(dmax * c.step <= 4096.f * xref)) return false;
  const bool lorentz = fmaf(xm, xm, c.y * c.y) >= kLorentzR2;
  const int ex = (__float_as_int(xref) >> 23) & 0xff;  // xref = m 2^(ex - 127), 1 <= m < 2
  const float sg = __int_as_float((254 - ex) << 23);   // 2^(127 - ex)
  const float sg2 = sg * sg;
  c.a *= sg;
  c.b *= sg;
  if (lorentz) {
    const float ys = c.y * sg;
    c.B1 = ys * ys;
    c.d = -1.f;
  } else {
    c.B1 *= sg2;
    c.d *= sg2 * sg2;
  }
  c.KA = c.K * (sg2 * sg2);
  c.K *= sg2;
  return true;
}

// Branch-free evaluation of one line at the lane's PTS points (fast class); lk[k] = lane + 32 k.
template <int KIND, int PTS>
__device__ __forceinline__ void eval_fast(const LineC& c, const float* lk, float* acc) {
  if (is_binned(KIND)) return;  // binned lines are never in the fast class
  const float4 f0 = *reinterpret_cast<const float4*>(&c.a);  // a, b, B1, d
  const float K = c.K;
  if (KIND == PXC_VOIGT) {
    // far wing, W4 region I: K (v + 1) / (v^2 + e), v = x^2 + c1 (five FP32 FMAs and one MUFU
    // reciprocal per point); no point of this warp is near the centre, so x = x(lane 0) + m step
    // keeps full relative accuracy
    const float KA = c.KA;  // K sigma^4, the rescaled numerator's constant term
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      const float x = fmaf(lk[k], f0.y, f0.x);
      const float v = fmaf(x, x, f0.z);
      acc[k] = fmaf(fmaf(v, K, KA), frcp(fmaf(v, v, f0.w)), acc[k]);
    }
  } else {
    // the line centre may lie among these points: x from the exact integer offset
    const float KG = c.KA;
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      const float x = fmaf(lk[k] + f0.x, f0.y, f0.w);
      if (is_pseudo_voigt(KIND)) {
        const float x2 = x * x;
        acc[k] = fmaf(K, frcp(x2 + 1.f), fmaf(KG, fex2(-x2), acc[k]));
      } else if (KIND == PXC_LORENTZ) {
        acc[k] = fmaf(K, frcp(fmaf(x, x, f0.z)), acc[k]);
      } else {
        acc[k] = fmaf(K, fex2(-(x * x)), acc[k]);
      }
    }
  }
}

// Two lines at once (more independent work per point, half the loop overhead).
template <int KIND, int PTS>
__device__ __forceinline__ void eval_fast2(const LineC& c, const LineC& e, const float* lk, float* acc) {
  if (is_binned(KIND)) return;
  if (KIND == PXC_VOIGT) {
    const float4 a0 = *reinterpret_cast<const float4*>(&c.a), a1 = *reinterpret_cast<const float4*>(&c.K);
    const float4 b0 = *reinterpret_cast<const float4*>(&e.a), b1 = *reinterpret_cast<const float4*>(&e.K);
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      const float x = fmaf(lk[k], a0.y, a0.x), y = fmaf(lk[k], b0.y, b0.x);
      const float u = fmaf(x, x, a0.z), v = fmaf(y, y, b0.z);
      const float du = fmaf(u, u, a0.w), dv = fmaf(v, v, b0.w);
      const float nu = fmaf(u, a1.x, a1.y), nv = fmaf(v, b1.x, b1.y);
      // n_u / d_u + n_v / d_v with one reciprocal (six FP32 operations and half a MUFU per point)
      acc[k] = fmaf(fmaf(nv, du, nu * dv), frcp(du * dv), acc[k]);
    }
  } else {
    eval_fast<KIND, PTS>(c, lk, acc);
    eval_fast<KIND, PTS>(e, lk, acc);
  }
}

// Lorentzian-limit Voigt lines from their 16-byte front records {a, b, sigma^2 y^2, K}.
template <int PTS>
__device__ __forceinline__ void eval_lor2(const LineC& c, const LineC& e, const float* lk, float* acc) {
  const float4 a = *reinterpret_cast<const float4*>(&c.a), b = *reinterpret_cast<const float4*>(&e.a);
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const float x = fmaf(lk[k], a.y, a.x), y = fmaf(lk[k], b.y, b.x);
    const float du = fmaf(x, x, a.z), dv = fmaf(y, y, b.z);
    acc[k] = fmaf(fmaf(b.w, du, a.w * dv), frcp(du * dv), acc[k]);
  }
}
template <int PTS>
__device__ __forceinline__ void eval_lor1(const LineC& c, const float* lk, float* acc) {
  const float4 a = *reinterpret_cast<const float4*>(&c.a);
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const float x = fmaf(lk[k], a.y, a.x);
    acc[k] = fmaf(a.w, frcp(fmaf(x, x, a.z)), acc[k]);
  }
}

// Binned profiles at the lane's PTS points inside the window (bin-centre offset t in the
// kind's unit, bin [t - h, t + h]):
//   Gaussian    mass = (erf(t + h) - erf(t - h)) / 2, from erfc of |t -+ h|: the difference of
//               the two erfc when both edges are on one side (no cancellation in the tails),
//               1 - (erfc + erfc) / 2 when the bin holds the centre
//   Lorentzian  mass = (atan(t + h) - atan(t - h)) / pi = atan2(2h, 1 + t^2 - h^2) / pi
//   Voigt       mean of the W4 Voigt over the bin by composite 2-point Gauss-Legendre on
//               subintervals of a quarter of the local scale (measured against the oracle's
//               adaptive quadrature: <= 7e-5 relative in FP64 over narrow-to-wide lines)
template <int KIND, int PTS>
__device__ __forceinline__ void eval_binned(const LineC& c, int wbase, int lane, float* acc) {
  constexpr int BASE = KIND & 3;
  const unsigned span = (unsigned)(c.hi - c.lo);
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const int b0 = wbase + 32 * k;
    if (b0 > c.hi || b0 + 31 < c.lo) continue;
    const int li = b0 + lane;
    const bool in = (unsigned)(li - c.lo) <= span;
    const float t = fmaf((float)li - c.pf, c.step, c.nfs);
    float v;
    if (BASE == PXC_LORENTZ) {
      v = c.K * atan2f(c.step, fmaf(t, t, c.B1));
    } else if (BASE == PXC_VOIGT) {
      // subintervals no wider than a quarter of the local scale: the larger width within six
      // widths of the centre, the distance to the centre beyond (at most 1024 per bin)
      const float dist = fmaxf(0.f, fabsf(t) - 0.5f * c.step);
      const float scale = dist < 6.f * c.d ? c.d : dist;
      const float nsf = fminf(fmaxf(ceilf(c.step * frcp(0.25f * scale)), 1.f), 1024.f);
      const int ns = (int)nsf;
      const float w = c.step * frcp(nsf);               // subinterval width
      const float gofs = 0.28867513459481287f * w;      // nodes at +-w / (2 sqrt 3)
      float x = fmaf(-0.5f, c.step, t) + 0.5f * w;      // first subinterval centre
      float sum = 0.f;
      for (int j = 0; j < ns; ++j) {
        sum += w4_re(x - gofs, c.y) + w4_re(x + gofs, c.y);
        x += w;
      }
      v = c.K * sum * (0.5f * frcp(nsf));
    } else {
      const float ta = t - c.B1, tb = t + c.B1;
      const float qa = erfcf(fabsf(ta)), qb = erfcf(fabsf(tb));
      const bool same = ta >= 0.f || tb <= 0.f;
      v = c.K * (same ? fabsf(qa - qb) : 2.f - qa - qb);
    }
    acc[k] += in ? v : 0.f;
  }
}

// Far-wing formula with a lane mask (the window ends among this warp's points).
template <int KIND, int PTS>
__device__ __forceinline__ void eval_fastmask(const LineC& c, int wbase, int lane, float* acc) {
  if (is_binned(KIND)) {
    eval_binned<KIND, PTS>(c, wbase, lane, acc);
    return;
  }
  const unsigned span = (unsigned)(c.hi - c.lo);
  const int rel0 = wbase + lane - c.lo;
  if (KIND == PXC_VOIGT) {
    const float x0 = fmaf((float)(wbase + lane) - c.pf, c.step, c.nfs);
    const float s32 = 32.f * c.step;
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      const float x = fmaf((float)k, s32, x0);
      const float v = region_one_or_direct(fmaf(x, x, c.B1), c.K, c.d, c.masks);
      acc[k] += (unsigned)(rel0 + 32 * k) <= span ? v : 0.f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
      const float x = fmaf((float)(wbase + lane + 32 * k) - c.pf, c.step, c.nfs);
      float v;
      if (is_pseudo_voigt(KIND)) {
        const float x2 = x * x;
        v = fmaf(c.K, frcp(x2 + 1.f), c.KA * fex2(-x2));
      } else {
        v = KIND == PXC_LORENTZ ? c.K * frcp(fmaf(x, x, c.B1)) : c.K * fex2(-(x * x));
      }
      acc[k] += (unsigned)(rel0 + 32 * k) <= span ? v : 0.f;
    }
  }
}

// Region II real rational Re w = y N(X) / D(X), X = x^2, coefficients from Y = y^2 (see
// eval_slow for the factored forms).
struct RegionII {
  float n0, n1, n2, n3, d0, d1, d2, d3;
};
__device__ __forceinline__ RegionII region2(float y) {
  const float bq = 0.5641896f;
  const float Y = y * y;
  RegionII r;
  r.n3 = bq;
  r.n2 = bq * (3.f * Y - 4.5f);
  r.n1 = bq * ((3.f * Y + 1.f) * Y + 5.25f);
  r.n0 = 0.125f * bq * (2.f * Y + 5.f) * ((4.f * Y + 12.f) * Y + 3.f);
  r.d3 = 4.f * Y - 6.f;
  r.d2 = (6.f * Y - 6.f) * Y + 10.5f;
  r.d1 = ((4.f * Y + 6.f) * Y + 9.f) * Y - 4.5f;
  r.d0 = (((Y + 6.f) * Y + 10.5f) * Y + 4.5f) * Y + 0.5625f;
  return r;
}

// Warps near the centre whose points all have |x| + y >= 5.5: the region II rational (W4's
// two-level continued fraction) where |x| + y < 15 and region I beyond, window edges masked.
template <int KIND, int PTS>
__device__ __forceinline__ void eval_mid(const LineC& c, int wbase, int lane, float* acc) {
  if (KIND != PXC_VOIGT) return;
  const unsigned span = (unsigned)(c.hi - c.lo);
  const int rel0 = wbase + lane - c.lo;
  const RegionII r = region2(c.y);
  const float Ky = c.Kc * c.y;
  const float x0 = fmaf((float)(wbase + lane) - c.pf, c.step, c.nfs);
  const float s32 = 32.f * c.step;
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const float x = fmaf((float)k, s32, x0);
    const float X = x * x;
    float v;
    if (!(c.masks & kRegion2Everywhere) && fabsf(x) + c.y >= 15.f) {  // region I: the quartic below
                                                                      // would overflow FP32 for very large x
      v = region_one_or_direct(X + c.B1, c.K, c.d, c.masks);
    } else {
      const float N = fmaf(fmaf(fmaf(r.n3, X, r.n2), X, r.n1), X, r.n0);
      const float D = fmaf(fmaf(fmaf(X + r.d3, X, r.d2), X, r.d1), X, r.d0);
      v = Ky * N * frcp(D);
    }
    acc[k] += (unsigned)(rel0 + 32 * k) <= span ? v : 0.f;
  }
}

// Warps near the line core (Voigt), some point with |x| + y < 5.5.  Points with |x| + y >= 5.5 take
// W4's region-II formula (region I instead beyond 15 when the warp's |x| reaches 1e4, where the
// region-II quartic would leave the FP32 range), the real rational
// Re w = y N(X) / D(X) in X = x^2 (N cubic, D monic quartic, coefficients from Y = y^2 once per line
// and warp; Humlicek's constants satisfy a = 2.5 b, which gives the factored forms of region2).
// Points with |x| + y < 5.5 take one formula per line where one
// suffices: for y <= 0.4 the region-IV form e^u - t P(u) / Q(u) over the whole disc (measured in
// FP32 against scipy's wofz: <= 4.8e-5 relative wherever Re w > 1e-6 of its peak, below W4's own
// region III/IV split, 9.1e-5), for y >= 0.9 the region-III rational (<= 3.8e-5; that whole disc
// is region III), and W4's region III/IV test per point in between.  A block then follows at most
// two paths instead of four.  With 8 or more points per lane, blocks of 32 points whose nearest
// point is beyond the region-I reach keep the region-I formula (a uniform branch).
template <int KIND, int PTS>
__device__ __forceinline__ void eval_slow(const LineC& c, int wbase, int lane, const float* lk, float* acc) {
  if (is_binned(KIND)) return;  // binned lines are never in the core class
  const unsigned span = (unsigned)(c.hi - c.lo);
  const RegionII r = region2(c.y);
  const float Ky = c.Kc * c.y;
  const int core = c.y <= 0.4f ? 4 : (c.y >= 0.9f ? 3 : 0);
#pragma unroll
  for (int k = 0; k < PTS; ++k) {
    const int b0 = wbase + 32 * k;
    if (b0 > c.hi || b0 + 31 < c.lo) continue;
    const int li = b0 + lane;
    const bool in = (unsigned)(li - c.lo) <= span;
    const float dmin = fmaxf(0.f, fmaxf(c.cen - (float)(b0 + 31), (float)b0 - c.cen));
    if (PTS >= 8 && dmin > c.reach) {
      // the whole block is in region I (uniform branch): the fast-path formula (measured to pay
      // off for wide warps only; narrow ones rarely have such blocks among their core lines)
      const float x = fmaf(lk[k], c.b, c.a);
      acc[k] += in ? region_one_or_direct(fmaf(x, x, c.B1), c.K, c.d, c.masks) : 0.f;
      continue;
    }
    const float x = fmaf((float)li - c.pf, c.step, c.nfs);
    const float sx = fabsf(x) + c.y;
    float v;
    if (sx >= 15.f && !(c.masks & kRegion2Everywhere)) {
      // region I (the region-II quartic in x^2 would leave the FP32 range for very large x)
      v = region_one_or_direct(fmaf(x, x, c.B1), c.K, c.d, c.masks);
    } else if (sx >= 5.5f) {
      const float X = x * x;
      const float N = fmaf(fmaf(fmaf(r.n3, X, r.n2), X, r.n1), X, r.n0);
      const float D = fmaf(fmaf(fmaf(X + r.d3, X, r.d2), X, r.d1), X, r.d0);
      v = Ky * N * frcp(D);
    } else if (core == 4) {
      v = c.Kc * w4_reg4_re(x, c.y);
    } else if (core == 3) {
      v = c.Kc * w4_reg3_re(x, c.y);
    } else {
      v = c.Kc * w4_core_re(x, c.y);
    }
    acc[k] += in ? v : 0.f;
  }
}

// Forward kernel.  The CTA's warps share kNB bulk-copy stage buffers of SL lines; each warp turns
// every staged record into its own line constants and class (so no CTA barrier is needed inside a
// work item), keeping two in-order lists in private shared memory.  From the front: the fast
// lines whose record is one float4 (Voigt: the Lorentzian-limit lines, evaluated in pairs with no
// per-pair test; other kinds: every fast line).  From the back: the rest (Voigt region-I fast
// lines, paired when adjacent, and the edge, mid and core classes).  The last warp to finish
// reading a stage buffer re-arms it with the copy kNB stages ahead, so warps drift apart by up to
// kNB - 1 stages instead of waiting for each other at every stage.
// Stage buffers per CTA: three for multi-warp CTAs (warps drift by up to two stages); two for
// one-warp CTAs, whose single warp never waits for another (the smaller shared-memory footprint
// lets more of them reside on an SM).
#ifndef PXC_STAGE_BUFFERS
#define PXC_STAGE_BUFFERS 3
#endif
#ifndef PXC_STAGE_BUFFERS_1W
#define PXC_STAGE_BUFFERS_1W 2
#endif
template <int THREADS>
constexpr int stage_buffers() { return THREADS == 32 ? PXC_STAGE_BUFFERS_1W : PXC_STAGE_BUFFERS; }

template <int THREADS, int SL>
constexpr size_t profile_smem() {
  return (size_t)stage_buffers<THREADS>() * SL * (16 + 8 + 4) + (size_t)(THREADS / 32) * SL * sizeof(LineC);
}

template <int KIND, int THREADS, int PTS, int SL, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_profile(const ProfP p) {
  constexpr int SEG = THREADS * PTS, WPTS = 32 * PTS, NW = THREADS / 32;
  constexpr int SBYTES = SL * (16 + 8 + 4);
  constexpr int kNB = stage_buffers<THREADS>();
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  unsigned char* raw = dyn_smem;                                              // [kNB][SBYTES]
  LineC* wl = reinterpret_cast<LineC*>(dyn_smem + kNB * SBYTES);             // [NW][SL]
  __shared__ __align__(8) uint64_t full[kNB];
  __shared__ int consumed[kNB];
  __shared__ int issued[kNB];
  __shared__ Item item_sh[2];
  __shared__ int abort_sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int wbase = warp * WPTS;
  float lk[PTS];  // lane + 32 k
#pragma unroll
  for (int k = 0; k < PTS; ++k) lk[k] = (float)(lane + 32 * k);
  const unsigned lt = (1u << lane) - 1u;
  LineC* my = wl + warp * SL;
  if (tid == 0) {
    for (int b = 0; b < kNB; ++b) { mbar_init(&full[b], 1); consumed[b] = 0; issued[b] = 0; }
    fence_mbar_init();
    abort_sh = 0;
  }
  __syncthreads();
  unsigned phase = 0;  // bit b: parity this warp waits for next on buffer b
  const unsigned long long n_items = *p.n_items;
  const float dnu_f = (float)p.dnu, nu_min_f = (float)p.nu_min;

  for (int iter = 0;; ++iter) {
    if (tid == 0) {
      unsigned long long it = atomicAdd(p.queue, 1ull);
      if (it < n_items && !abort_sh) item_sh[iter & 1] = p.items[it]; else item_sh[iter & 1].cond = -1;
    }
    __syncthreads();  // also: every warp has finished the previous item, so all stage buffers are free
    const Item item = item_sh[iter & 1];
    if (item.cond < 0) break;
    const CondDev cd = p.cond[item.cond];
    const int64_t i0 = (int64_t)item.seg * SEG;
    const float* Is = p.Is + (int64_t)cd.slot * p.is_stride;
    const int j0 = item.begin & ~3;
    const int nst = item.end > item.begin ? (item.end - j0 + SL - 1) / SL : 0;

    float sum[PTS];
#pragma unroll
    for (int k = 0; k < PTS; ++k) sum[k] = 0.f;

    auto issue = [&](int st) {
      const int b = st % kNB;
      const int64_t J = (int64_t)j0 + (int64_t)st * SL;
      unsigned char* dst = raw + b * SBYTES;
      issued[b] += 1;
      mbar_expect_tx(&full[b], SBYTES);
      bulk_g2s(dst, p.pos + J, SL * 16, &full[b]);
      bulk_g2s(dst + SL * 16, p.par + J, SL * 8, &full[b]);
      bulk_g2s(dst + SL * 24, Is + J, SL * 4, &full[b]);
    };
    if (tid == 0) {
      fence_proxy_async();
      for (int st = 0; st < kNB && st < nst; ++st) issue(st);
    }

    bool aborted = false;
    for (int st = 0; st < nst; ++st) {
      const int b = st % kNB;
      const bool ok = mbar_wait_bounded(&full[b], (phase >> b) & 1u, p.spin_limit);
      phase ^= 1u << b;
      if (__any_sync(0xffffffffu, !ok)) { aborted = true; break; }
      // this warp's constants and classes for the staged lines, compacted in line order
      const unsigned char* src = raw + b * SBYTES;
      int nf = 0, no = 0;
#pragma unroll
      for (int r = 0; r < SL / 32; ++r) {
        const int j = lane + 32 * r;
        const int64_t J = (int64_t)j0 + (int64_t)st * SL + j;
        const float is = reinterpret_cast<const float*>(src + SL * 24)[j];
        const bool live = is != 0.f && J >= item.begin && J < item.end;
        // lines whose FP32 scaled intensity is zero add nothing: a round of 32 without a live line
        // builds no constants (lists far below their strongest line are mostly such lines)
        if (!__any_sync(0xffffffffu, live)) continue;
        const int4 p4 = reinterpret_cast<const int4*>(src)[j];
        const float2 pr = reinterpret_cast<const float2*>(src + SL * 16)[j];
        LineC c;
        line_constants<KIND, SEG>(p4, pr, is, cd, i0, wbase, dnu_f, nu_min_f, live, c);
        int cls = line_class<KIND, WPTS>(c, wbase);
        if (KIND == PXC_VOIGT && cls == 1 && !scale_for_pairs<WPTS>(c, wbase)) cls = 2;
        c.masks = cls;
        // unscaled region-I terms of this line and warp: the direct form unless |x| or y reaches
        // 1e9 somewhere in the warp (then u^2 could leave the FP32 range)
        if (KIND == PXC_VOIGT && cls >= 2) {
          const float dmax = fmaxf(fabsf(c.cen - (float)wbase), fabsf(c.cen - (float)(wbase + WPTS - 1)));
          if (dmax * c.step > 1e9f || c.y > 1e9f) c.masks |= kWideRange;
          if (dmax * c.step < 1e4f && c.y < 15.f) c.masks |= kRegion2Everywhere;
        }
        // front: lines whose fast record is one float4 (Voigt: the Lorentzian limit {a, b, s^2 y^2, K};
        // other kinds: every fast line); back: Voigt region-I fast lines and the other classes
        const bool front = cls == 1 && (KIND != PXC_VOIGT || c.d < 0.f);
        const unsigned bf = __ballot_sync(0xffffffffu, front);
        const unsigned bo = __ballot_sync(0xffffffffu, cls >= 1 && !front);
        if (front) {
          if (KIND == PXC_VOIGT) *reinterpret_cast<float4*>(&my[nf + __popc(bf & lt)]) = make_float4(c.a, c.b, c.B1, c.K);
          else my[nf + __popc(bf & lt)] = c;
        }
        if (cls >= 1 && !front) my[SL - 1 - (no + __popc(bo & lt))] = c;
        nf += __popc(bf);
        no += __popc(bo);
      }
      __syncwarp();
      // release the stage buffer; the last warp re-arms it
      if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&consumed[b], 1) == NW - 1) {
          consumed[b] = 0;
          __threadfence_block();
          if (st + kNB < nst) {
            fence_proxy_async();
            issue(st + kNB);
          }
        }
      }
      float acc[PTS];
#pragma unroll
      for (int k = 0; k < PTS; ++k) acc[k] = 0.f;
      int i = 0;
      if (KIND == PXC_VOIGT) {
        for (; i + 1 < nf; i += 2) eval_lor2<PTS>(my[i], my[i + 1], lk, acc);
        if (i < nf) eval_lor1<PTS>(my[i], lk, acc);
      } else {
        for (; i + 1 < nf; i += 2) eval_fast2<KIND, PTS>(my[i], my[i + 1], lk, acc);
        if (i < nf) eval_fast<KIND, PTS>(my[i], lk, acc);
      }
      for (int q = SL - 1; q >= SL - no; --q) {
        const LineC& c = my[q];
        const int cls = c.masks & 7;
        if (KIND == PXC_VOIGT && cls == 1) {
          if (q - 1 >= SL - no && (my[q - 1].masks & 7) == 1) {
            eval_fast2<KIND, PTS>(c, my[q - 1], lk, acc);
            --q;
          } else {
            eval_fast<KIND, PTS>(c, lk, acc);
          }
        } else if (cls == 2) eval_fastmask<KIND, PTS>(c, wbase, lane, acc);
        else if (cls == 4) eval_mid<KIND, PTS>(c, wbase, lane, acc);
        else eval_slow<KIND, PTS>(c, wbase, lane, lk, acc);
      }
#pragma unroll
      for (int k = 0; k < PTS; ++k) sum[k] += acc[k];
      __syncwarp();
    }
    if (aborted) {
      if (lane == 0) { atomicOr(p.err, ERRB_TIMEOUT); abort_sh = 1; }
    } else {
#pragma unroll
      for (int k = 0; k < PTS; ++k) {
        const int li = wbase + lane + 32 * k;
        const int64_t gi = i0 + li;
        if (item.slot < 0) {
          if (gi < p.n_grid) {
            float* o = p.sigma + (int64_t)item.cond * p.n_grid + gi;
            if (p.accumulate) { if (nst) *o += sum[k]; } else *o = sum[k];
          }
        } else {
          p.partial[(int64_t)item.slot * SEG + li] = sum[k];
        }
      }
    }
  }
  // after a timeout, let copies already issued land before the CTA leaves (bounded again)
  __syncthreads();
  if (tid == 0 && abort_sh) {
    for (int b = 0; b < kNB; ++b)
      if (issued[b] > 0) mbar_wait_bounded(&full[b], (unsigned)((issued[b] - 1) & 1), p.drain_limit);
  }
}

// Compiled tile configurations: {threads, points per lane, lines per stage, min CTAs per SM}.
// Segment widths 128, 256, 1024 and 2048 points.  (One-warp tiles of 256 and 512 points, with
// fewer line-warp constant builds per evaluation, measured slower than tile 0 on the 1e9-line
// list: 12.4 and 17.9 against 11.4 ms per 1e8-line call.)
#ifndef PXC_TILE0_SL
#define PXC_TILE0_SL 64
#endif
#ifndef PXC_TILE0_PTS
#define PXC_TILE0_PTS 4
#define PXC_TILE0_MINB 32
#endif
#define PXC_TILES(X) \
  X(0, 32, PXC_TILE0_PTS, PXC_TILE0_SL, PXC_TILE0_MINB) X(1, 64, 4, 64, 16) X(2, 128, 8, 64, 6) X(3, 128, 16, 128, 4)

int tile_seg(int tile) {
#define X(i, T, P, S, M) if (tile == i) return T * P;
  PXC_TILES(X)
#undef X
  return 0;
}

template <int KIND, int T, int P, int S, int M>
static int occupancy_one() {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_profile<KIND, T, P, S, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)profile_smem<T, S>());
    attr = true;
  }
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_profile<KIND, T, P, S, M>, T, profile_smem<T, S>());
  return n > 0 ? n : 1;
}

template <int KIND>
static int occupancy_kind(int tile) {
#define X(i, T, P, S, M) if (tile == i) return occupancy_one<KIND, T, P, S, M>();
  PXC_TILES(X)
#undef X
  return 1;
}

int profile_occupancy(int kind, int tile) {
  switch (kind) {
    case PXC_GAUSS_DOPPLER: return occupancy_kind<PXC_GAUSS_DOPPLER>(tile);
    case PXC_GAUSS_HWHM: return occupancy_kind<PXC_GAUSS_HWHM>(tile);
    case PXC_LORENTZ: return occupancy_kind<PXC_LORENTZ>(tile);
    case PXC_BINNED_GAUSS_DOPPLER: return occupancy_kind<PXC_BINNED_GAUSS_DOPPLER>(tile);
    case PXC_BINNED_GAUSS_HWHM: return occupancy_kind<PXC_BINNED_GAUSS_HWHM>(tile);
    case PXC_BINNED_LORENTZ: return occupancy_kind<PXC_BINNED_LORENTZ>(tile);
    case PXC_BINNED_VOIGT: return occupancy_kind<PXC_BINNED_VOIGT>(tile);
    case PXC_PV_THOMPSON: return occupancy_kind<PXC_PV_THOMPSON>(tile);
    case PXC_PV_OLIVERO: return occupancy_kind<PXC_PV_OLIVERO>(tile);
    case PXC_PV_LIULIN: return occupancy_kind<PXC_PV_LIULIN>(tile);
    default: return occupancy_kind<PXC_VOIGT>(tile);
  }
}

template <int KIND>
static void launch_kind(const ProfP& p, int tile, int grid_ctas, cudaStream_t s) {
#define X(i, T, P, S, M) \
  if (tile == i) { k_profile<KIND, T, P, S, M><<<grid_ctas, T, profile_smem<T, S>(), s>>>(p); return; }
  PXC_TILES(X)
#undef X
}

void launch_profile(const ProfP& p, int tile, int grid_ctas, cudaStream_t s) {
  switch (p.kind) {
    case PXC_GAUSS_DOPPLER: launch_kind<PXC_GAUSS_DOPPLER>(p, tile, grid_ctas, s); break;
    case PXC_GAUSS_HWHM: launch_kind<PXC_GAUSS_HWHM>(p, tile, grid_ctas, s); break;
    case PXC_LORENTZ: launch_kind<PXC_LORENTZ>(p, tile, grid_ctas, s); break;
    case PXC_BINNED_GAUSS_DOPPLER: launch_kind<PXC_BINNED_GAUSS_DOPPLER>(p, tile, grid_ctas, s); break;
    case PXC_BINNED_GAUSS_HWHM: launch_kind<PXC_BINNED_GAUSS_HWHM>(p, tile, grid_ctas, s); break;
    case PXC_BINNED_LORENTZ: launch_kind<PXC_BINNED_LORENTZ>(p, tile, grid_ctas, s); break;
    case PXC_BINNED_VOIGT: launch_kind<PXC_BINNED_VOIGT>(p, tile, grid_ctas, s); break;
    case PXC_PV_THOMPSON: launch_kind<PXC_PV_THOMPSON>(p, tile, grid_ctas, s); break;
    case PXC_PV_OLIVERO: launch_kind<PXC_PV_OLIVERO>(p, tile, grid_ctas, s); break;
    case PXC_PV_LIULIN: launch_kind<PXC_PV_LIULIN>(p, tile, grid_ctas, s); break;
    default: launch_kind<PXC_VOIGT>(p, tile, grid_ctas, s); break;
  }
  note_launches(1);
}

// ------------------------------------------------------------------ wavelength grids
// Eq. (xsec) sampled on a wavelength grid (Sec. 2.4.3): lambda_i = lambda_min + i dlambda,
// nu_i = U / lambda_i.  Each line's position in grid steps is (U/nu_l - lambda_min)/dlambda =
// ic + f (FP64 in the preparation pass), so the offset from the line centre is
//   nu_i - nu_l = U (lambda_l - lambda_i) / (lambda_i lambda_l) = ((ic - i) + f) (U dlambda / lambda_l) / lambda_i
// with the integer difference exact in FP32 and no cancellation between nearly equal wavenumbers.
// A CTA of kSegWl threads takes one work item (a segment and its line range) at a time, thread j
// owning point i0 + j; the lines' constants are built once per staged line (thread q builds line q
// of the stage) and every thread adds the lines whose window holds its point.  The Voigt kind
// evaluates Humlicek's W4 in every region; the pseudo-Voigts a Lorentzian and a Gaussian.
struct LineWl {
  int ic, lo, hi, ok;
  float f, kd;     // position fraction; U dlambda / lambda_l (cm^-1 per grid step at lambda_i = lambda_l)
  float s, y;      // Gauss/Voigt: 1/(s sqrt2) = sqrt(ln2)/alpha and y; Lorentz: gamma; pseudo-Voigt: 1/h
  float K, K2;     // amplitudes (pseudo-Voigt: Lorentzian and Gaussian parts)
};

template <int KIND>
__device__ __forceinline__ LineWl line_constants_wl(const int4 p4, const float2 pr, float is, const CondDev& cd,
                                                    const ProfP& p, bool valid) {
  LineWl c;
  c.ic = p4.x;
  c.f = __int_as_float(p4.y);
  c.lo = p4.z;
  c.hi = p4.w;
  const double lam_l = p.nu_min + ((double)c.ic + (double)c.f) * p.dnu;
  const float nu = (float)(p.wl_unit / lam_l);
  c.kd = (float)(p.wl_unit * p.dnu / lam_l);
  const float g = pr.x * exp2f(pr.y * cd.log2_tratio) * cd.P_f;
  c.ok = valid && is != 0.f && c.lo <= c.hi;
  if (KIND == PXC_LORENTZ) {
    const float gm = fmaxf(g, kGammaMin);
    c.s = gm;
    c.y = gm * gm;
    c.K = is * gm * kInvPi;
    c.K2 = 0.f;
    return c;
  }
  const float alpha = fmaxf(KIND == PXC_GAUSS_HWHM ? cd.hwhm : cd.alpha_coef * nu,
                            is_pseudo_voigt(KIND) ? kAlphaMinWide : kAlphaMin);
  if (is_pseudo_voigt(KIND)) {
    float G, wl, wg;
    pv_params<KIND>(alpha, g, &G, &wl, &wg);
    const float ih = 2.f / G;
    c.s = ih;
    c.y = 0.f;
    c.K = is * wl * kInvPi * ih;
    c.K2 = is * wg * (kSqrtLn2 * kInvSqrtPi) * ih;
    return c;
  }
  const float cc = kSqrtLn2 / alpha;
  c.s = cc;
  c.y = KIND == PXC_VOIGT ? g * cc : 0.f;
  c.K = is * cc * kInvSqrtPi;
  c.K2 = 0.f;
  return c;
}

template <int KIND>
__device__ __forceinline__ float eval_wl(const LineWl& c, float dnu_pt) {
  if (KIND == PXC_LORENTZ) return c.K * frcp(fmaf(dnu_pt, dnu_pt, c.y));
  if (is_pseudo_voigt(KIND)) {
    const float t = dnu_pt * c.s, t2 = t * t;
    return fmaf(c.K, frcp(t2 + 1.f), c.K2 * fex2(-t2));
  }
  const float x = dnu_pt * c.s;
  if (KIND == PXC_VOIGT) return c.K * w4_re(x, c.y);
  return c.K * __expf(-x * x);
}

template <int KIND>
__global__ void __launch_bounds__(kSegWl) k_profile_wl(const ProfP p) {
  __shared__ LineWl sl[kSegWl];
  const unsigned long long n_items = *p.n_items;
  for (unsigned long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    const Item item = p.items[it];
    const CondDev cd = p.cond[item.cond];
    const float* Is = p.Is + (int64_t)cd.slot * p.is_stride;
    const int64_t gi = (int64_t)item.seg * kSegWl + threadIdx.x;
    const float inv_lam = (float)(1.0 / (p.nu_min + (double)gi * p.dnu));
    float sum = 0.f;
    for (int j0 = item.begin; j0 < item.end; j0 += kSegWl) {
      const int n = min(kSegWl, item.end - j0);
      __syncthreads();  // the previous stage's constants are no longer read
      if ((int)threadIdx.x < n) {
        const int j = j0 + (int)threadIdx.x;
        sl[threadIdx.x] = line_constants_wl<KIND>(p.pos[j], p.par[j], Is[j], cd, p, true);
      }
      __syncthreads();
      float stage = 0.f;
      for (int q = 0; q < n; ++q) {
        const LineWl& c = sl[q];
        if (!c.ok || gi < c.lo || gi > c.hi) continue;
        const float dnu_pt = ((float)(c.ic - (int)gi) + c.f) * c.kd * inv_lam;
        stage += eval_wl<KIND>(c, dnu_pt);
      }
      sum += stage;
    }
    if (gi < p.n_grid) {
      float* o = p.sigma + (int64_t)item.cond * p.n_grid + gi;
      if (item.slot < 0) {
        if (p.accumulate) { if (item.end > item.begin) *o += sum; } else *o = sum;
      } else {
        p.partial[(int64_t)item.slot * kSegWl + threadIdx.x] = sum;
      }
    }
  }
}

void launch_profile_wl(const ProfP& p, int64_t max_items, cudaStream_t s) {
  int64_t blocks = max_items < 148 * 16 ? max_items : 148 * 16;
  if (blocks < 1) blocks = 1;
  switch (p.kind) {
    case PXC_GAUSS_DOPPLER: k_profile_wl<PXC_GAUSS_DOPPLER><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
    case PXC_GAUSS_HWHM: k_profile_wl<PXC_GAUSS_HWHM><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
    case PXC_LORENTZ: k_profile_wl<PXC_LORENTZ><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
    case PXC_PV_THOMPSON: k_profile_wl<PXC_PV_THOMPSON><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
    case PXC_PV_OLIVERO: k_profile_wl<PXC_PV_OLIVERO><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
    case PXC_PV_LIULIN: k_profile_wl<PXC_PV_LIULIN><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
    default: k_profile_wl<PXC_VOIGT><<<(unsigned)blocks, kSegWl, 0, s>>>(p); break;
  }
  note_launches(1);
}

// ------------------------------------------------------------------ adjoint
// Each warp takes batches of 32 sorted lines, strided across the warps.  Lane q loads line q and
// builds its widths; for each line of the batch in turn the lanes stride over its window (the
// line's values broadcast by shuffles), recompute the profile and its width derivatives at each
// point and accumulate them against w = dL/dsigma_s; a butterfly sum leaves the totals in every
// lane and lane q keeps line q's.  With G = sum w f, Da = sum w df/dalpha, Dg = sum w df/dgamma (times the scaled intensity
// I_s) the chain rule gives
//   dL/dA_l = I_s G / A_l,  dL/dgamma_ref_l = I_s (T_ref/T)^n P Dg,
//   per-line shares of dL/dT (T_rot), dL/dT_vib and dL/dP (FP64, reduced in a fixed order),
// evaluated on all 32 lanes at once (one line each).
// Voigt: f = (c/sqrt(pi)) Re w(z), z = (x + i gamma) c, c = sqrt(ln2)/alpha, with
//   df/dgamma = -(c^2/sqrt(pi)) Im w'(z),  df/dalpha = -(c/(alpha sqrt(pi))) (Re w + Re(z w'(z))).
template <int KIND>
__global__ void __launch_bounds__(256) k_adjoint(const AdjP p) {
  const int lane = threadIdx.x & 31;
  const int64_t n = (int64_t)*p.n_dev;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const float dnu_f = (float)p.dnu;
  // warp gw takes lines gw, gw + W, gw + 2W, ... (W warps), 32 of them per batch: lines that crowd
  // one wavenumber (consecutive in the sorted order) spread over many warps
  for (int64_t b0 = gw; b0 < n; b0 += 32 * warps) {
    const int64_t j = b0 + (int64_t)lane * warps;
    const bool valid = j < n;
    int4 p4 = make_int4(0, 0, 0, -1);
    float2 pr = make_float2(0.f, 0.f);
    float is = 0.f;
    if (valid) {
      p4 = p.pos[j];
      pr = p.par[j];
      is = p.Is[j];
    }
    const int ic = p4.x;
    const float f = __int_as_float(p4.y);
    const float nu_f = (float)(p.nu_min + ((double)ic + (double)f) * p.dnu);
    const float alpha = fmaxf(KIND == PXC_GAUSS_HWHM ? p.cond.hwhm : p.cond.alpha_coef * nu_f, kAlphaMinWide);
    const float gfac = exp2f(pr.y * p.cond.log2_tratio) * p.cond.P_f;   // dgamma/dgamma_ref
    const float gam = KIND == PXC_LORENTZ ? fmaxf(pr.x * gfac, kGammaMin) : KIND == PXC_VOIGT ? pr.x * gfac : 0.f;
    const float cc = kSqrtLn2 / alpha;
    float g0 = 0.f, ga = 0.f, gg = 0.f;  // lane q: the sums of line q
    for (int q = 0; q < 32; ++q) {
      if (__shfl_sync(0xffffffffu, is, q) == 0.f) continue;  // no contribution to sigma (uniform)
      const int icq = __shfl_sync(0xffffffffu, ic, q);
      const int loq = __shfl_sync(0xffffffffu, p4.z, q), hiq = __shfl_sync(0xffffffffu, p4.w, q);
      const float fq = __shfl_sync(0xffffffffu, f, q);
      const float ccq = __shfl_sync(0xffffffffu, cc, q), gamq = __shfl_sync(0xffffffffu, gam, q);
      float s0 = 0.f, sa = 0.f, sg = 0.f;
      for (int i = loq + lane; i <= hiq; i += 32) {
        const float wi = p.w[i];
        const float x = ((float)(i - icq) - fq) * dnu_f;
        if (KIND == PXC_VOIGT) {
          const float X = x * ccq, Y = gamq * ccq;
          cplx w, dw;
          w4_full(X, Y, &w, &dw);
          s0 = fmaf(wi, w.r, s0);
          sg = fmaf(wi, dw.i, sg);
          sa = fmaf(wi, w.r + (X * dw.r - Y * dw.i), sa);
        } else if (KIND == PXC_LORENTZ) {
          const float x2 = x * x, g2 = gamq * gamq;
          const float d = 1.f / (x2 + g2);
          s0 = fmaf(wi, d, s0);
          sg = fmaf(wi, (x2 - g2) * d * d, sg);
        } else {
          const float X = x * ccq;
          const float e = expf(-X * X);
          s0 = fmaf(wi, e, s0);
          sa = fmaf(wi, e * X * X, sa);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
      }
      if (lane == q) {
        g0 = s0;
        ga = sa;
        gg = sg;
      }
    }
    if (!valid) continue;
    if (is == 0.f) {
      // zero scaled intensity: no contribution to sigma, hence none to any gradient
      p.lineT[j] = 0.0;
      p.lineTv[j] = 0.0;
      p.lineP[j] = 0.0;
      continue;
    }
    const uint32_t t = p.sidx[j];
    double G = 0.0, Da = 0.0, Dg = 0.0;
    const double ccd = cc, ad = alpha, spi = 1.7724538509055160273;
    if (KIND == PXC_VOIGT) {
      G = ccd / spi * g0;
      Dg = -(ccd * ccd / spi) * gg;
      Da = -(ccd / (ad * spi)) * ga;
    } else if (KIND == PXC_LORENTZ) {
      G = (double)gam / kPi * g0;
      Dg = gg / kPi;
    } else {
      G = ccd / spi * g0;
      Da = ccd / spi * (-(double)g0 + 2.0 * ga) / ad;
    }
    const double I = is;
    const double A = p.sA[j];
    if (p.dA) p.dA[t] = (float)(I * G / A);
    if (p.dgref) p.dgref[t] = (float)(I * (double)gfac * Dg);
    const int32_t u = p.su[j], l = p.sl[j];
    const double Eu = p.srec[u].x, El = p.srec[l].x;
    const double c2 = p.c2, T = p.T;
    const double Q = p.qres[0], dQ = p.qres[1], dQv = p.qres[2];
    double dlnT, dlnTv = 0.0;
    if (p.T_vib > 0.0) {
      const double evl = p.E_vib[l], evu = p.E_vib[u];
      const double erl = El - evl, eru = Eu - evu;
      const double nv = evu - evl, nr = eru - erl;
      const double X = c2 * (nv / p.T_vib + nr / T);
      const double st = 1.0 / expm1(X);
      dlnT = c2 * erl / (T * T) - c2 * nr / (T * T) * st - dQ / Q;
      dlnTv = c2 * evl / (p.T_vib * p.T_vib) - c2 * nv / (p.T_vib * p.T_vib) * st - dQv / Q;
    } else {
      const double nu = Eu - El;
      const double st = 1.0 / expm1(c2 * nu / T);
      dlnT = c2 * El / (T * T) - c2 * nu / (T * T) * st - dQ / Q;
    }
    const bool dop = KIND == PXC_GAUSS_DOPPLER || KIND == PXC_VOIGT;
    const bool pres = KIND == PXC_LORENTZ || KIND == PXC_VOIGT;
    const double dadT = dop ? ad / (2.0 * T) : 0.0;
    const double dgdT = pres ? -(double)pr.y * (double)gam / T : 0.0;
    const double dgdP = pres ? (double)gam / p.P : 0.0;
    p.lineT[j] = I * (dlnT * G + dadT * Da + dgdT * Dg);
    p.lineTv[j] = I * dlnTv * G;
    p.lineP[j] = I * dgdP * Dg;
  }
}

void launch_adjoint(const AdjP& p, cudaStream_t s) {
  int64_t blocks = ((p.n_max + 31) / 32 * 32 + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  switch (p.kind) {
    case PXC_GAUSS_DOPPLER: k_adjoint<PXC_GAUSS_DOPPLER><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    case PXC_GAUSS_HWHM: k_adjoint<PXC_GAUSS_HWHM><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    case PXC_LORENTZ: k_adjoint<PXC_LORENTZ><<<(unsigned)blocks, 256, 0, s>>>(p); break;
    default: k_adjoint<PXC_VOIGT><<<(unsigned)blocks, 256, 0, s>>>(p); break;
  }
  note_launches(1);
}

// Fixed-order FP64 reduction of the per-line scalar shares in two launches: kRedBlocks CTAs each
// sum one contiguous range (thread t takes every kRedThreads-th element of it, then a fixed tree),
// and one CTA sums the per-CTA totals the same way.  The order depends only on the line count.
constexpr int kRedBlocks = 296, kRedThreads = 256;

__device__ __forceinline__ void tree3(double (*r)[kRedThreads], double* sa, double* sb, double* sc) {
  const int t = threadIdx.x;
  r[0][t] = *sa;
  r[1][t] = *sb;
  r[2][t] = *sc;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (t < o) {
      r[0][t] += r[0][t + o];
      r[1][t] += r[1][t + o];
      r[2][t] += r[2][t + o];
    }
    __syncthreads();
  }
  *sa = r[0][0];
  *sb = r[1][0];
  *sc = r[2][0];
}

__global__ void __launch_bounds__(kRedThreads) k_adjoint_reduce(const double* __restrict__ a,
                                                                const double* __restrict__ b,
                                                                const double* __restrict__ c,
                                                                const unsigned long long* __restrict__ n_dev,
                                                                double* __restrict__ part) {
  __shared__ double r[3][kRedThreads];
  const int64_t n = (int64_t)*n_dev;
  const int64_t per = (n + kRedBlocks - 1) / kRedBlocks;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  double sa = 0.0, sb = 0.0, sc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
    sa += a[i];
    sb += b[i];
    sc += c[i];
  }
  tree3(r, &sa, &sb, &sc);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sa;
    part[kRedBlocks + blockIdx.x] = sb;
    part[2 * kRedBlocks + blockIdx.x] = sc;
  }
}

__global__ void __launch_bounds__(kRedThreads) k_adjoint_reduce_final(const double* __restrict__ part, double* oa,
                                                                      double* ob, double* oc) {
  __shared__ double r[3][kRedThreads];
  double sa = 0.0, sb = 0.0, sc = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) {
    sa += part[i];
    sb += part[kRedBlocks + i];
    sc += part[2 * kRedBlocks + i];
  }
  tree3(r, &sa, &sb, &sc);
  if (threadIdx.x == 0) {
    if (oa) *oa = sa;
    if (ob) *ob = sb;
    if (oc) *oc = sc;
  }
}

size_t adjoint_reduce_scratch_bytes() { return (size_t)3 * kRedBlocks * sizeof(double); }

void launch_adjoint_reduce(const double* lineT, const double* lineTv, const double* lineP,
                           const unsigned long long* n_dev, double* scratch, double* outT, double* outTv,
                           double* outP, cudaStream_t s) {
  k_adjoint_reduce<<<kRedBlocks, kRedThreads, 0, s>>>(lineT, lineTv, lineP, n_dev, scratch);
  k_adjoint_reduce_final<<<1, kRedThreads, 0, s>>>(scratch, outT, outTv, outP);
  note_launches(2);
}

}  // namespace pxc
