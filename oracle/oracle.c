/*
 * FP64 CPU ORACLE for line intensities and cross sections (PyExoCross 2.0,
 * Secs. 2.4.2, 2.4.3, 3.1, 3.2).  TEST INFRASTRUCTURE ONLY: imported by the
 * tests, by the smoke check and by the CPU-baseline leg of the benchmark, never
 * by the product path.  It shares no code, header or constant table with the
 * CUDA library; the only thing both consume is the seeded input data.
 *
 * Everything here is the plain definition, written out loop by loop in double
 * precision, in the paper's order:
 *   Q(T)                 Eq. (pf):          sum_n g_n exp(-c2 E_n / T)
 *   Q(T_vib, T_rot)      Eq. (Q nlte 2T):   sum g exp(-c2 E_vib/T_vib) exp(-c2 E_rot/T_rot)
 *   nu                   Sec. 2.4.3:        E' - E'', lines with nu <= 0 discarded
 *   I (LTE)              Eq. (abs intensity lte)
 *   I (two-temperature)  Eqs. (nlte v), (nlte ab 2T)  [brace reading R9 below]
 *   sigma(nu_i)          Eq. (xsec):        sum_l I_l f_l(nu_i - nu_l), |nu_i - nu_l| <= cut
 *   profiles             Table (profile): Doppler/Gaussian, Lorentzian, Voigt
 *   adjoint              analytic derivatives of the above (no counterpart in the paper)
 *   Q(T_rot), densities  Eq. (Q nlte Nvib): sum g n_vib exp(-c2 E_rot / T_rot)
 *   I (vibronic density) Eq. (nlte ab pop density)
 *   epsilon (emission)   Eqs. (ems intensity lte), (nlte em 2T), (nlte em pop density)
 *   W(T)                 Eq. (cf), cooling function  [reading R17 below for non-LTE]
 *   binned profiles      Table (profile), binned Doppler / Gaussian / Lorentzian / Voigt [R19]
 *   pseudo-Voigts        Table (profile), Thompson, Olivero and Liu-Lin pseudo-Voigt [R20]
 *
 * Readings where the text is silent or garbled:
 *   R7  nu = E' - E''; lines with nu <= 0 are dropped (nu = 0 would divide by zero).
 *   R8  window of grid indices: i_lo = ceil((nu - cut - nu_min)/dnu),
 *       i_hi = floor((nu + cut - nu_min)/dnu), plain IEEE double, no FMA,
 *       clamped to the grid; no renormalisation of the truncated profile.
 *   R9  2T stimulated-emission factor 1 - exp(-c2 (nu_vib/T_vib + nu_rot/T_rot)).
 *   R10 threshold: keep |I| >= S_min.  Two-temperature populations can be inverted
 *       (I < 0, gain); such lines are kept, not silently dropped.
 *   R11 line order: ascending nu bit pattern, ties by transition index.
 *   R12 per-list exponent: k = frexp exponent of max kept I; I_s = (float) ldexp(I, -k).
 *   R15 states with NaN energy are absent: skipped in Q, lines touching them dropped.
 *   R17 the cooling function is the sum of the emission intensities of all lines
 *       with nu > 0 (no grid window, no threshold); Eq. (cf) is its LTE case, and the
 *       non-LTE populations of Eqs. (nlte em 2T) / (nlte em pop density) give the
 *       non-LTE cases.
 *   R19 a binned profile is the average of the profile over the grid bin centred on the grid
 *       point, (1/dnu) int_{nu_i - dnu/2}^{nu_i + dnu/2} f(nu - nu_l) dnu; the window (R8) is
 *       the same as for sampled profiles.  Gaussian: erf/erfc differences; Lorentzian: the
 *       arctangent difference; Voigt (no closed-form integral): adaptive Gauss-Legendre
 *       quadrature of the Voigt profile over the bin to 1e-12 relative.
 *   R20 pseudo-Voigt profiles (Table profile names them and cites their sources; the paper prints
 *       no formula): f = eta L(x; G/2) + (1 - eta) G(x; G/2) (Liu-Lin: c_L L + c_G G), a Lorentzian
 *       and a Gaussian of one common full width G, from the Gaussian and Lorentzian full widths
 *       fG = 2 alpha, fL = 2 gamma of the Voigt kind:
 *         Thompson (Thompson, Cox, Hastings 1987): G^5 = fG^5 + 2.69269 fG^4 fL + 2.42843 fG^3 fL^2
 *           + 4.47163 fG^2 fL^3 + 0.07842 fG fL^4 + fL^5, eta = 1.36603 r - 0.47719 r^2 + 0.11116 r^3,
 *           r = fL / G;
 *         Olivero (Olivero, Longbothum 1977): the Voigt width G = 0.5346 fL + sqrt(0.2166 fL^2 + fG^2)
 *           with the same mixing eta(fL / G) (reading: the paper names only the width formula);
 *         Liu-Lin (Liu, Lin et al. 2001): d = (fL - fG)/(fL + fG), G = (fL + fG)(1 - 0.18121 (1 - d^2)
 *           - (0.023665 e^{0.6 d} + 0.00418 e^{-1.9 d}) sin(pi d)), c_L = 0.68188 + 0.61293 d
 *           - 0.18384 d^2 - 0.11568 d^3, c_G = 0.32460 - 0.61825 d + 0.17681 d^2 + 0.12109 d^3.
 *       The Kielkopf and Di Rocco-Cruzado variants the table also names are not written: their
 *       coefficients are in publications this restatement could not consult.
 *   R21 wavelength grids (Sec. 2.4.3: spectra in wavenumber, or in wavelength in nm or um): a
 *       grid uniform in wavelength, lambda_i = lambda_min + i dlambda in a unit with
 *       nu = U / lambda (U = 1e7 for nm, 1e4 for um); sigma is sampled at nu_i = U / lambda_i and
 *       the cut-off stays in cm^-1.  |nu_i - nu_l| <= cut is U/(nu_l + cut) <= lambda_i <=
 *       U/(nu_l - cut), so the window is i_lo = ceil((U/(nu + cut) - lambda_min)/dlambda),
 *       i_hi = floor((U/(nu - cut) - lambda_min)/dlambda) (the last point when nu <= cut), plain
 *       IEEE double, clamped; lines are ordered by descending nu (ascending wavelength), ties by
 *       transition index, so windows stay monotone along the order.  Sampled profiles only.
 *   R18 vibronic densities: E_rot = E - E_vib within each manifold, T (the condition's
 *       temperature) is T_rot, and the densities are used as given (every formula is
 *       invariant under a common scale, so normalising them changes nothing).
 *   Doppler HWHM alpha = (nu/c) sqrt(2 N_A k_B T ln2 / M) (standard form; the
 *   formula itself is deferred by the paper to its predecessor).
 *   Lorentz HWHM gamma = gamma_ref (T_ref/T)^n P, with P used directly in the
 *   unit of gamma_ref.  In the two-temperature case T_rot sets both widths
 *   (Sec. 3.3).
 *
 * Voigt: V(x) = Re w(z) / (s sqrt(2 pi)), s = alpha / sqrt(2 ln 2),
 * z = (x + i gamma) / (s sqrt 2), the definition behind scipy.special.voigt_profile
 * (Table "profile").  w(z) is evaluated by the Laplace continued fraction
 * (40 levels) for |x| + y >= 8 and by Weideman's rational expansion
 * (J.A.C. Weideman, SIAM J. Numer. Anal. 31 (1994) 1497, N = 64, coefficients
 * from the trapezoidal Fourier sum of (L^2 + t^2) exp(-t^2) at t = L tan(theta/2))
 * elsewhere.  Pinned in the tests against scipy.special.wofz / voigt_profile.
 *
 * Status codes: 0 ok, 1 bad argument, 2 state id out of range, 3 non-finite
 * input, 4 Boltzmann exponent overflow (> 709.78).
 */
#include <complex.h>
#undef I
#define CI _Complex_I
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 exact SI values, in cgs (Table "notation"). */
#define ORC_H 6.62607015e-27     /* erg s */
#define ORC_C 2.99792458e10      /* cm / s */
#define ORC_KB 1.380649e-16      /* erg / K */
#define ORC_NA 6.02214076e23     /* 1 / mol */
#define ORC_PI 3.14159265358979323846
#define ORC_LN2 0.69314718055994530942
#define ORC_SQRTPI 1.77245385090551602730
#define ORC_EXP_MAX 709.78

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_ID = 2, ORC_ERR_NONFINITE = 3, ORC_ERR_OVERFLOW = 4 };
enum { ORC_GAUSS_DOPPLER = 0, ORC_GAUSS_HWHM = 1, ORC_LORENTZ = 2, ORC_VOIGT = 3 };
/* Binned kinds (Table profile): kind | ORC_BINNED, the widths of the base kind kind & 3. */
enum { ORC_BINNED = 4 };
/* Pseudo-Voigt kinds (R20), sampled, with the widths of the Voigt kind. */
enum { ORC_PV_THOMPSON = 8, ORC_PV_OLIVERO = 9, ORC_PV_LIULIN = 10 };

double orc_c2(void) { return ORC_H * ORC_C / ORC_KB; }

/* Threads of the OpenMP loops (the CPU-baseline timing reports all cores and one). */
void orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }

/* ---------------------------------------------------------------------------
 * Faddeeva function w(z), Im z >= 0.
 * ------------------------------------------------------------------------ */

#define WEID_N 64
static double weid_a[WEID_N + 1];
static double weid_L;

static void weideman_init(void) {
  /* f(t) = (L^2 + t^2) exp(-t^2) expanded in powers of Z = e^{i theta},
   * t = L tan(theta/2); a_n = (1/2pi) int f cos(n theta) dtheta by the
   * trapezoidal rule on 2M points (f = 0 at theta = +-pi), M = 2N. */
  const int M = 2 * WEID_N;
  weid_L = sqrt((double)WEID_N / sqrt(2.0));
  for (int n = 0; n <= WEID_N; ++n) {
    double s = 0.0;
    for (int k = -M + 1; k <= M - 1; ++k) {
      double th = (double)k * ORC_PI / (double)M;
      double t = weid_L * tan(0.5 * th);
      s += exp(-t * t) * (weid_L * weid_L + t * t) * cos((double)n * th);
    }
    weid_a[n] = s / (2.0 * (double)M);
  }
}

__attribute__((constructor)) static void orc_init(void) { weideman_init(); }

static double complex faddeeva(double x, double y) {
  double complex z = x + CI * y;
  if (fabs(x) + y >= 8.0) {
    /* w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...)))) */
    double complex r = 0.0;
    for (int k = 40; k >= 1; --k) r = (0.5 * (double)k) / (z - r);
    return (CI / ORC_SQRTPI) / (z - r);
  }
  double complex d = weid_L - CI * z;
  double complex Z = (weid_L + CI * z) / d;
  double complex p = 0.0;
  for (int n = WEID_N; n >= 1; --n) p = p * Z + weid_a[n];
  return 2.0 * p / (d * d) + (1.0 / ORC_SQRTPI) / d;
}

void orc_faddeeva(int64_t n, const double* x, const double* y, double* re, double* im) {
  for (int64_t i = 0; i < n; ++i) {
    double complex w = faddeeva(x[i], y[i]);
    re[i] = creal(w);
    im[i] = cimag(w);
  }
}

/* ---------------------------------------------------------------------------
 * Profiles f(x) with x = nu_i - nu_l, and their width derivatives.
 * ------------------------------------------------------------------------ */

static double prof_gauss(double x, double a) {
  return sqrt(ORC_LN2 / ORC_PI) / a * exp(-ORC_LN2 * x * x / (a * a));
}
static double prof_lorentz(double x, double g) { return g / (ORC_PI * (x * x + g * g)); }
static double prof_voigt(double x, double a, double g) {
  double s = a / sqrt(2.0 * ORC_LN2);
  double complex w = faddeeva(x / (s * sqrt(2.0)), g / (s * sqrt(2.0)));
  return creal(w) / (s * sqrt(2.0 * ORC_PI));
}

static double prof_pseudo_voigt(int kind, double x, double a, double g);  /* R20, below */

/* f, df/dalpha, df/dgamma for one profile kind. */
static void prof_eval(int kind, double x, double a, double g, double* f, double* fa, double* fg) {
  if (kind == ORC_GAUSS_DOPPLER || kind == ORC_GAUSS_HWHM) {
    double v = prof_gauss(x, a);
    *f = v;
    *fa = v * (-1.0 / a + 2.0 * ORC_LN2 * x * x / (a * a * a));
    *fg = 0.0;
  } else if (kind == ORC_LORENTZ) {
    double d = x * x + g * g;
    *f = prof_lorentz(x, g);
    *fa = 0.0;
    *fg = (x * x - g * g) / (ORC_PI * d * d);
  } else {
    /* V = Re w(z) c / sqrt(pi), c = sqrt(ln2)/alpha = 1/(s sqrt 2), z = (x + i g) c.
     * w'(z) = -2 z w(z) + 2i/sqrt(pi).
     * dV/dgamma = -(c^2/sqrt(pi)) Im w'(z);
     * dV/dalpha = -(c/(alpha sqrt(pi))) (Re w + Re(z w'(z))). */
    double c = sqrt(ORC_LN2) / a;
    double complex z = (x + CI * g) * c;
    double complex w = faddeeva(creal(z), cimag(z));
    double complex wp = -2.0 * z * w + 2.0 * CI / ORC_SQRTPI;
    *f = creal(w) * c / ORC_SQRTPI;
    *fg = -(c * c / ORC_SQRTPI) * cimag(wp);
    *fa = -(c / (a * ORC_SQRTPI)) * (creal(w) + creal(z * wp));
  }
}

void orc_profile(int kind, int64_t n, const double* x, double a, double g, double* f, double* fa, double* fg) {
  if (kind >= ORC_PV_THOMPSON) {  /* forward only */
    for (int64_t i = 0; i < n; ++i) {
      f[i] = prof_pseudo_voigt(kind, x[i], a, g);
      if (fa) fa[i] = 0.0;
      if (fg) fg[i] = 0.0;
    }
    return;
  }
  for (int64_t i = 0; i < n; ++i) {
    double t0, t1, t2;
    prof_eval(kind, x[i], a, g, &t0, &t1, &t2);
    f[i] = t0;
    if (fa) fa[i] = t1;
    if (fg) fg[i] = t2;
  }
}

/* ---------------------------------------------------------------------------
 * Binned profiles (R19).  x is the offset of the bin centre from the line centre.
 * ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
static double gl_x[2][16], gl_w[2][16];
static int gl_ready = 0;
static void gl_init(void) {
  const int ns[2] = {8, 16};
  for (int q = 0; q < 2; ++q) {
    int n = ns[q];
    for (int i = 0; i < n; ++i) {
      double x = cos(ORC_PI * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      double dp = n * (x * p1 - p0) / (x * x - 1.0);
      gl_x[q][i] = x;
      gl_w[q][i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
  }
  gl_ready = 1;
}

static double gl_voigt(int q, double a, double b, double alpha, double g) {
  const int n = q ? 16 : 8;
  double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
  for (int i = 0; i < n; ++i) s += gl_w[q][i] * prof_voigt(m + h * gl_x[q][i], alpha, g);
  return s * h;
}

/* Integral of the Voigt profile over [a, b]: accept the 16-point rule where it agrees with the
 * 8-point rule to the absolute tolerance tol (1e-13 of the whole bin's first estimate),
 * otherwise bisect (at most 30 levels). */
static double adapt_voigt(double a, double b, double alpha, double g, double tol, int depth) {
  double i8 = gl_voigt(0, a, b, alpha, g), i16 = gl_voigt(1, a, b, alpha, g);
  if (fabs(i16 - i8) <= tol || depth >= 30) return i16;
  double m = 0.5 * (a + b);
  return adapt_voigt(a, m, alpha, g, tol, depth + 1) + adapt_voigt(m, b, alpha, g, tol, depth + 1);
}

static double integrate_voigt(double a, double b, double alpha, double g) {
  double tol = 1e-13 * fabs(gl_voigt(1, a, b, alpha, g)) + 1e-300;
  return adapt_voigt(a, b, alpha, g, tol, 0);
}

/* Average over the bin [x - dnu/2, x + dnu/2] of the base profile kind & 3. */
static double prof_binned(int kind, double x, double dnu, double a, double g) {
  double lo = x - 0.5 * dnu, hi = x + 0.5 * dnu;
  int base = kind & 3;
  if (base == ORC_LORENTZ) {
    /* atan(tb) - atan(ta) = atan((tb - ta) / (1 + ta tb)) (+ pi when 1 + ta tb < 0) */
    double ta = lo / g, tb = hi / g, p = 1.0 + ta * tb;
    double d = atan((tb - ta) / p) + (p < 0.0 ? ORC_PI : 0.0);
    return d / (ORC_PI * dnu);
  }
  if (base == ORC_VOIGT) {
    if (!gl_ready) gl_init();
    if (lo < 0.0 && hi > 0.0)   /* split at the line centre, where the profile peaks */
      return (integrate_voigt(lo, 0.0, a, g) + integrate_voigt(0.0, hi, a, g)) / dnu;
    return integrate_voigt(lo, hi, a, g) / dnu;
  }
  /* Gaussian: mass = (erf(tb) - erf(ta)) / 2, t = u sqrt(ln2) / alpha; erfc on one side */
  double c = sqrt(ORC_LN2) / a, ta = lo * c, tb = hi * c, mass;
  if (ta >= 0.0) mass = 0.5 * (erfc(ta) - erfc(tb));
  else if (tb <= 0.0) mass = 0.5 * (erfc(-tb) - erfc(-ta));
  else mass = 0.5 * (erf(tb) - erf(ta));
  return mass / dnu;
}

/* Pseudo-Voigt (R20) from the Doppler and Lorentz HWHMs a, g: the common full width G and the
 * weights of the Lorentzian and the Gaussian. */
static void pv_params(int kind, double a, double g, double* G, double* wl, double* wg) {
  const double fG = 2.0 * a, fL = 2.0 * g;
  if (kind == ORC_PV_LIULIN) {
    const double d = (fL - fG) / (fL + fG);
    *G = (fL + fG) * (1.0 - 0.18121 * (1.0 - d * d) -
                      (0.023665 * exp(0.6 * d) + 0.00418 * exp(-1.9 * d)) * sin(ORC_PI * d));
    *wl = 0.68188 + d * (0.61293 + d * (-0.18384 + d * -0.11568));
    *wg = 0.32460 + d * (-0.61825 + d * (0.17681 + d * 0.12109));
    return;
  }
  if (kind == ORC_PV_THOMPSON) {
    const double s5 = pow(fG, 5) + 2.69269 * pow(fG, 4) * fL + 2.42843 * pow(fG, 3) * fL * fL +
                      4.47163 * fG * fG * pow(fL, 3) + 0.07842 * fG * pow(fL, 4) + pow(fL, 5);
    *G = pow(s5, 0.2);
  } else {
    *G = 0.5346 * fL + sqrt(0.2166 * fL * fL + fG * fG);
  }
  const double r = fL / *G;
  *wl = r * (1.36603 + r * (-0.47719 + r * 0.11116));
  *wg = 1.0 - *wl;
}

static double prof_pseudo_voigt(int kind, double x, double a, double g) {
  double G, wl, wg;
  pv_params(kind, a, g, &G, &wl, &wg);
  const double h = 0.5 * G;
  return wl * prof_lorentz(x, h) + wg * prof_gauss(x, h);
}

void orc_pv_params(int kind, int64_t n, const double* a, const double* g, double* G, double* wl, double* wg) {
  for (int64_t i = 0; i < n; ++i) pv_params(kind, a[i], g[i], &G[i], &wl[i], &wg[i]);
}

/* Profile value at a grid point: sampled (kinds 0..3), bin-averaged (kinds 4..7) or a
 * pseudo-Voigt (kinds 8..10). */
static double prof_point(int kind, double x, double dnu, double a, double g) {
  if (kind >= ORC_PV_THOMPSON) return prof_pseudo_voigt(kind, x, a, g);
  if (kind & ORC_BINNED) return prof_binned(kind, x, dnu, a, g);
  if (kind == ORC_LORENTZ) return prof_lorentz(x, g);
  if (kind == ORC_VOIGT) return prof_voigt(x, a, g);
  return prof_gauss(x, a);
}

void orc_profile_binned(int kind, int64_t n, const double* x, double dnu, double a, double g, double* f) {
  if (!gl_ready) gl_init();
  for (int64_t i = 0; i < n; ++i) f[i] = prof_binned(kind | ORC_BINNED, x[i], dnu, a, g);
}

/* ---------------------------------------------------------------------------
 * Partition functions, Eqs. (pf) and (Q nlte 2T).  T_vib <= 0 selects LTE.
 * out[0] = Q, out[1] = dQ/dT (LTE) or dQ/dT_rot (2T), out[2] = dQ/dT_vib (2T).
 * ------------------------------------------------------------------------ */

int orc_partition(const double* E, const int32_t* g, const double* E_vib, int64_t n,
                  double T, double T_vib, double* out) {
  if (!(T > 0.0) || (T_vib > 0.0 && !E_vib)) return ORC_ERR_ARG;
  const double c2 = orc_c2();
  double Q = 0.0, dQ = 0.0, dQv = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    if (isnan(E[s])) continue;
    if (!isfinite(E[s])) return ORC_ERR_NONFINITE;
    if (T_vib > 0.0) {
      double ev = E_vib[s], er = E[s] - ev;
      if (!isfinite(ev)) return ORC_ERR_NONFINITE;
      double xv = -c2 * ev / T_vib, xr = -c2 * er / T;
      if (xv + xr > ORC_EXP_MAX || xv > ORC_EXP_MAX || xr > ORC_EXP_MAX) return ORC_ERR_OVERFLOW;
      double term = (double)g[s] * exp(xv) * exp(xr);
      Q += term;
      dQ += term * c2 * er / (T * T);
      dQv += term * c2 * ev / (T_vib * T_vib);
    } else {
      double x = -c2 * E[s] / T;
      if (x > ORC_EXP_MAX) return ORC_ERR_OVERFLOW;
      double term = (double)g[s] * exp(x);
      Q += term;
      dQ += term * c2 * E[s] / (T * T);
    }
  }
  out[0] = Q;
  out[1] = dQ;
  out[2] = dQv;
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Per-line quantities.  For every transition t:
 *   nu[t]  = E[u] - E[l]                       (NaN if a state is absent)
 *   I[t]   = intensity in cm/molecule (0 where not kept)
 *   keep[t]= 1 if nu > 0, the cut-off window meets the grid, and I >= S_min
 *   ilo/ihi= window of grid indices (R8), valid where keep
 * A is float64 (A_f32 == 0) or float32.
 * ------------------------------------------------------------------------ */

static int window(double nu, double nu_min, double dnu, int64_t n_grid, double cut, double wl_unit,
                  int64_t* lo, int64_t* hi) {
  double a, b;
  if (wl_unit > 0.0) {  /* R21: nu_min, dnu are lambda_min, dlambda */
    a = ceil((wl_unit / (nu + cut) - nu_min) / dnu);
    b = nu - cut > 0.0 ? floor((wl_unit / (nu - cut) - nu_min) / dnu) : (double)(n_grid - 1);
  } else {
    a = ceil(((nu - cut) - nu_min) / dnu);
    b = floor(((nu + cut) - nu_min) / dnu);
  }
  if (b < 0.0 || a > (double)(n_grid - 1) || a > b) return 0;
  *lo = a < 0.0 ? 0 : (int64_t)a;
  *hi = b > (double)(n_grid - 1) ? n_grid - 1 : (int64_t)b;
  return 1;
}

int orc_line_intensities(const double* E, const int32_t* g, const double* E_vib, int64_t n_states,
                         const int32_t* upper, const int32_t* lower, const void* A, int A_f32, int64_t n,
                         double T, double T_vib, double Q,
                         double nu_min, double dnu, int64_t n_grid, double cut, double threshold, double wl_unit,
                         double* nu_out, double* I_out, uint8_t* keep, int64_t* ilo, int64_t* ihi) {
  if (!(T > 0.0) || !(Q > 0.0) || !(dnu > 0.0) || cut < 0.0 || n_grid < 1) return ORC_ERR_ARG;
  const double c2 = orc_c2();
  int status = ORC_OK;
  for (int64_t t = 0; t < n; ++t) {
    int64_t u = upper[t], l = lower[t];
    nu_out[t] = NAN; I_out[t] = 0.0; keep[t] = 0; ilo[t] = 0; ihi[t] = -1;
    if (u < 0 || u >= n_states || l < 0 || l >= n_states) return ORC_ERR_ID;
    double a = A_f32 ? (double)((const float*)A)[t] : ((const double*)A)[t];
    if (!isfinite(a)) return ORC_ERR_NONFINITE;
    double nu = E[u] - E[l];
    nu_out[t] = nu;
    if (!(nu > 0.0)) continue;                                  /* R7, R15 */
    int64_t lo, hi;
    if (!window(nu, nu_min, dnu, n_grid, cut, wl_unit, &lo, &hi)) continue;
    double gu = (double)g[u];
    double pref = gu * a / (8.0 * ORC_PI * ORC_C * nu * nu);
    double I;
    if (T_vib > 0.0) {
      /* Eqs. (nlte v), (nlte ab 2T) */
      double ev_l = E_vib[l], er_l = E[l] - ev_l;
      double ev_u = E_vib[u], er_u = E[u] - ev_u;
      double nu_vib = ev_u - ev_l, nu_rot = er_u - er_l;
      double xv = -c2 * ev_l / T_vib, xr = -c2 * er_l / T;
      if (xv > ORC_EXP_MAX || xr > ORC_EXP_MAX || xv + xr > ORC_EXP_MAX) { status = ORC_ERR_OVERFLOW; break; }
      I = pref * exp(xv) * exp(xr) * (1.0 - exp(-c2 * (nu_vib / T_vib + nu_rot / T))) / Q;
    } else {
      /* Eq. (abs intensity lte) */
      double x = -c2 * E[l] / T;
      if (x > ORC_EXP_MAX) { status = ORC_ERR_OVERFLOW; break; }
      I = pref * exp(x) * (1.0 - exp(-c2 * nu / T)) / Q;
    }
    if (!(fabs(I) >= threshold)) continue;                      /* R10 */
    I_out[t] = I;
    keep[t] = 1;
    ilo[t] = lo;
    ihi[t] = hi;
  }
  return status;
}

/* ---------------------------------------------------------------------------
 * Population model of a state (the factor multiplying g in Q and in the intensities):
 *   LTE      exp(-c2 E / T)                                   Eq. (pf)
 *   2T       exp(-c2 E_vib / T_vib) exp(-c2 E_rot / T_rot)    Eq. (Q nlte 2T)
 *   density  n_vib exp(-c2 E_rot / T_rot)                     Eq. (Q nlte Nvib), R18
 * Selected by n_vib != NULL (density, needs E_vib), else T_vib > 0 (2T), else LTE.
 * Returns ORC_ERR_OVERFLOW when an exponent exceeds the double range.
 * ------------------------------------------------------------------------ */
static int population(const double* E, const double* E_vib, const double* n_vib, int64_t s, double T,
                      double T_vib, double* out) {
  const double c2 = orc_c2();
  if (n_vib) {
    double x = -c2 * (E[s] - E_vib[s]) / T;
    if (x > ORC_EXP_MAX) return ORC_ERR_OVERFLOW;
    *out = n_vib[s] * exp(x);
  } else if (T_vib > 0.0) {
    double xv = -c2 * E_vib[s] / T_vib, xr = -c2 * (E[s] - E_vib[s]) / T;
    if (xv > ORC_EXP_MAX || xr > ORC_EXP_MAX || xv + xr > ORC_EXP_MAX) return ORC_ERR_OVERFLOW;
    *out = exp(xv) * exp(xr);
  } else {
    double x = -c2 * E[s] / T;
    if (x > ORC_EXP_MAX) return ORC_ERR_OVERFLOW;
    *out = exp(x);
  }
  return ORC_OK;
}

/* Partition function with vibronic densities, Eq. (Q nlte Nvib): Q = sum g n_vib
 * exp(-c2 E_rot / T_rot); out[0] = Q, out[1] = dQ/dT_rot. */
int orc_partition_density(const double* E, const int32_t* g, const double* E_vib, const double* n_vib,
                          int64_t n, double T_rot, double* out) {
  if (!(T_rot > 0.0) || !E_vib || !n_vib) return ORC_ERR_ARG;
  const double c2 = orc_c2();
  double Q = 0.0, dQ = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    if (isnan(E[s])) continue;
    if (!isfinite(E[s]) || !isfinite(E_vib[s]) || !isfinite(n_vib[s])) return ORC_ERR_NONFINITE;
    double p;
    int st = population(E, E_vib, n_vib, s, T_rot, 0.0, &p);
    if (st) return st;
    double term = (double)g[s] * p;
    Q += term;
    dQ += term * c2 * (E[s] - E_vib[s]) / (T_rot * T_rot);
  }
  out[0] = Q;
  out[1] = dQ;
  return ORC_OK;
}

/* Absorption (emission == 0) or emission (emission == 1) intensities of every line under
 * the population model above, with the same selection as orc_line_intensities (nu > 0,
 * window on the grid, |value| >= threshold):
 *   absorption, LTE      Eq. (abs intensity lte)
 *   absorption, 2T       Eqs. (nlte v), (nlte ab 2T)      [R9]
 *   absorption, density  Eq. (nlte ab pop density): g' A n''_vib exp(-c2 E''_rot/T_rot)
 *                        (1 - exp(-c2 nu / T_rot)) / (8 pi c nu^2 Q)
 *   emission, LTE        Eq. (ems intensity lte):   g' h c A nu exp(-c2 E'/T) / (4 pi Q)
 *   emission, 2T         Eq. (nlte em 2T)
 *   emission, density    Eq. (nlte em pop density)
 * in cm/molecule (absorption) or erg/s/sr/molecule (emission).  Q is the model's own
 * partition function. */
int orc_intensities(int emission, const double* E, const int32_t* g, const double* E_vib, const double* n_vib,
                    int64_t n_states, const int32_t* upper, const int32_t* lower, const void* A, int A_f32, int64_t n,
                    double T, double T_vib, double Q, double nu_min, double dnu, int64_t n_grid, double cut,
                    double threshold, double wl_unit, double* nu_out, double* I_out, uint8_t* keep, int64_t* ilo,
                    int64_t* ihi) {
  if (!(T > 0.0) || !(Q > 0.0) || !(dnu > 0.0) || cut < 0.0 || n_grid < 1) return ORC_ERR_ARG;
  if ((n_vib || T_vib > 0.0) && !E_vib) return ORC_ERR_ARG;
  if (n_vib && T_vib > 0.0) return ORC_ERR_ARG;
  const double c2 = orc_c2();
  for (int64_t t = 0; t < n; ++t) {
    int64_t u = upper[t], l = lower[t];
    nu_out[t] = NAN; I_out[t] = 0.0; keep[t] = 0; ilo[t] = 0; ihi[t] = -1;
    if (u < 0 || u >= n_states || l < 0 || l >= n_states) return ORC_ERR_ID;
    double a = A_f32 ? (double)((const float*)A)[t] : ((const double*)A)[t];
    if (!isfinite(a)) return ORC_ERR_NONFINITE;
    double nu = E[u] - E[l];
    nu_out[t] = nu;
    if (!(nu > 0.0)) continue;                                  /* R7, R15 */
    int64_t lo, hi;
    if (!window(nu, nu_min, dnu, n_grid, cut, wl_unit, &lo, &hi)) continue;
    double val, p;
    int st;
    if (emission) {
      if ((st = population(E, E_vib, n_vib, u, T, T_vib, &p))) return st;
      val = (double)g[u] * ORC_H * ORC_C * a * nu * p / (4.0 * ORC_PI * Q);
    } else if (n_vib) {
      if ((st = population(E, E_vib, n_vib, l, T, T_vib, &p))) return st;
      val = (double)g[u] * a * p * (1.0 - exp(-c2 * nu / T)) / (8.0 * ORC_PI * ORC_C * nu * nu * Q);
    } else {
      double ev_l = 0.0, ev_u = 0.0;
      if (T_vib > 0.0) { ev_l = E_vib[l]; ev_u = E_vib[u]; }
      if ((st = population(E, E_vib, NULL, l, T, T_vib, &p))) return st;
      double stim = T_vib > 0.0 ? 1.0 - exp(-c2 * ((ev_u - ev_l) / T_vib + ((E[u] - ev_u) - (E[l] - ev_l)) / T))
                                : 1.0 - exp(-c2 * nu / T);
      val = (double)g[u] * a * p * stim / (8.0 * ORC_PI * ORC_C * nu * nu * Q);
    }
    if (!(fabs(val) >= threshold)) continue;                    /* R10 */
    I_out[t] = val;
    keep[t] = 1;
    ilo[t] = lo;
    ihi[t] = hi;
  }
  return ORC_OK;
}

/* Cooling function, Eq. (cf) and reading R17: W = sum over lines with nu > 0 of
 * g' h c A nu p(upper) / (4 pi Q), in erg/s/molecule/sr. */
int orc_cooling_function(const double* E, const int32_t* g, const double* E_vib, const double* n_vib,
                         int64_t n_states, const int32_t* upper, const int32_t* lower, const void* A, int A_f32,
                         int64_t n, double T, double T_vib, double Q, double* W_out) {
  if (!(T > 0.0) || !(Q > 0.0)) return ORC_ERR_ARG;
  if ((n_vib || T_vib > 0.0) && !E_vib) return ORC_ERR_ARG;
  double W = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    int64_t u = upper[t], l = lower[t];
    if (u < 0 || u >= n_states || l < 0 || l >= n_states) return ORC_ERR_ID;
    double a = A_f32 ? (double)((const float*)A)[t] : ((const double*)A)[t];
    if (!isfinite(a)) return ORC_ERR_NONFINITE;
    double nu = E[u] - E[l];
    if (!(nu > 0.0)) continue;
    double p;
    int st = population(E, E_vib, n_vib, u, T, T_vib, &p);
    if (st) return st;
    W += (double)g[u] * ORC_H * ORC_C * a * nu * p / (4.0 * ORC_PI * Q);
  }
  *W_out = W;
  return ORC_OK;
}

/* R12: k = exponent of the largest kept |intensity| (max = m 2^k, 0.5 <= m < 1). */
int32_t orc_list_exponent(const double* I, const uint8_t* keep, int64_t n) {
  double mx = 0.0;
  for (int64_t t = 0; t < n; ++t)
    if (keep[t] && fabs(I[t]) > mx) mx = fabs(I[t]);
  if (mx == 0.0) return 0;
  int k;
  frexp(mx, &k);
  return (int32_t)k;
}

void orc_scale_intensities(const double* I, const uint8_t* keep, int64_t n, int32_t k, float* I_s) {
  for (int64_t t = 0; t < n; ++t) I_s[t] = keep[t] ? (float)ldexp(I[t], -k) : 0.0f;
}

/* R11: kept lines in ascending (nu bit pattern, index) order; on a wavelength grid (R21) in
 * descending nu bit pattern, ties by ascending index. */
static const double* g_sort_nu;
static int g_sort_desc;
static int cmp_line(const void* pa, const void* pb) {
  int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  uint64_t ka, kb;
  memcpy(&ka, &g_sort_nu[a], 8);
  memcpy(&kb, &g_sort_nu[b], 8);
  if (ka != kb) return (ka < kb) != g_sort_desc ? -1 : 1;
  return a < b ? -1 : (a > b);
}

int64_t orc_sorted_order(const double* nu, const uint8_t* keep, int64_t n, double wl_unit, int64_t* perm) {
  int64_t m = 0;
  for (int64_t t = 0; t < n; ++t)
    if (keep[t]) perm[m++] = t;
  g_sort_nu = nu;
  g_sort_desc = wl_unit > 0.0;
  qsort(perm, (size_t)m, sizeof(int64_t), cmp_line);
  return m;
}

/* Grid point i as a wavenumber: nu_min + i dnu, or U / (lambda_min + i dlambda) (R21). */
static double grid_nu(double g0, double dg, int64_t i, double wl_unit) {
  return wl_unit > 0.0 ? wl_unit / (g0 + (double)i * dg) : g0 + (double)i * dg;
}

/* Segment binning: for grid segments [s*S, (s+1)*S), the first sorted line whose
 * window reaches the segment and one past the last whose window starts in or
 * before it.  Windows are monotone in nu, so the lines of a segment are
 * contiguous in sorted order. */
void orc_segment_ranges(const int64_t* ilo_sorted, const int64_t* ihi_sorted, int64_t m,
                        int64_t n_grid, int64_t S, int64_t* first, int64_t* last) {
  int64_t nseg = (n_grid + S - 1) / S;
  for (int64_t s = 0; s < nseg; ++s) {
    int64_t a = s * S, b = (s + 1) * S - 1;
    int64_t f = 0;
    while (f < m && ihi_sorted[f] < a) ++f;
    int64_t e = f;
    while (e < m && ilo_sorted[e] <= b) ++e;
    first[s] = f;
    last[s] = e;
  }
}

/* ---------------------------------------------------------------------------
 * Line widths (HWHM) for one condition.
 * ------------------------------------------------------------------------ */

void orc_widths(int kind, const double* nu, const float* gamma_ref, const float* n_T, int64_t n,
                double T, double P, double mass_da, double hwhm, double T_ref,
                double* alpha, double* gamma) {
  double dop = sqrt(2.0 * ORC_NA * ORC_KB * T * ORC_LN2 / mass_da) / ORC_C;
  /* binned kinds take the widths of their base kind, pseudo-Voigts those of the Voigt kind */
  kind = kind >= ORC_PV_THOMPSON ? ORC_VOIGT : (kind & 3);
  for (int64_t t = 0; t < n; ++t) {
    alpha[t] = kind == ORC_GAUSS_HWHM ? hwhm : nu[t] * dop;
    gamma[t] = (kind == ORC_LORENTZ || kind == ORC_VOIGT)
                   ? (double)gamma_ref[t] * pow(T_ref / T, (double)n_T[t]) * P
                   : 0.0;
  }
}

/* ---------------------------------------------------------------------------
 * Cross section, Eq. (xsec): sigma_i = sum_l I_l f_l(nu_i - nu_l) over the
 * window of each kept line.  Grid points nu_i = nu_min + i dnu.  The grid is
 * split among threads; each point sums its lines in transition-index order.
 * ------------------------------------------------------------------------ */

int orc_cross_section(int kind, const double* nu, const double* I, const double* alpha, const double* gamma,
                      const uint8_t* keep, const int64_t* ilo, const int64_t* ihi, int64_t n,
                      double nu_min, double dnu, int64_t n_grid, double wl_unit, double* sigma) {
  if (wl_unit > 0.0 && (kind & ORC_BINNED) && kind < ORC_PV_THOMPSON) return ORC_ERR_ARG;
  if (!gl_ready) gl_init();
  for (int64_t i = 0; i < n_grid; ++i) sigma[i] = 0.0;
  int64_t nblk = 256;
  int64_t bs = (n_grid + nblk - 1) / nblk;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t b = 0; b < nblk; ++b) {
    int64_t a0 = b * bs, a1 = a0 + bs - 1;
    if (a1 > n_grid - 1) a1 = n_grid - 1;
    if (a0 > a1) continue;
    for (int64_t t = 0; t < n; ++t) {
      if (!keep[t] || ihi[t] < a0 || ilo[t] > a1) continue;
      int64_t lo = ilo[t] > a0 ? ilo[t] : a0, hi = ihi[t] < a1 ? ihi[t] : a1;
      for (int64_t i = lo; i <= hi; ++i) {
        double x = grid_nu(nu_min, dnu, i, wl_unit) - nu[t];
        sigma[i] += I[t] * prof_point(kind, x, dnu, alpha[t], gamma[t]);
      }
    }
  }
  return ORC_OK;
}

/* The same sum on the grid points i0 .. i0+m-1 only (sampled checks at full size).  As in
 * orc_cross_section, the points are split among threads and each point sums its lines in
 * transition-index order. */
int orc_cross_section_window(int kind, const double* nu, const double* I, const double* alpha, const double* gamma,
                             const uint8_t* keep, const int64_t* ilo, const int64_t* ihi, int64_t n,
                             double nu_min, double dnu, int64_t i0, int64_t m, double wl_unit, double* sigma) {
  if (wl_unit > 0.0 && (kind & ORC_BINNED) && kind < ORC_PV_THOMPSON) return ORC_ERR_ARG;
  if (!gl_ready) gl_init();
  for (int64_t j = 0; j < m; ++j) sigma[j] = 0.0;
  int64_t nblk = m < 64 ? m : 64;
  if (nblk < 1) return ORC_OK;
  int64_t bs = (m + nblk - 1) / nblk;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t b = 0; b < nblk; ++b) {
    int64_t a0 = i0 + b * bs, a1 = a0 + bs - 1;
    if (a1 > i0 + m - 1) a1 = i0 + m - 1;
    if (a0 > a1) continue;
    for (int64_t t = 0; t < n; ++t) {
      if (!keep[t] || ihi[t] < a0 || ilo[t] > a1) continue;
      int64_t lo = ilo[t] > a0 ? ilo[t] : a0, hi = ihi[t] < a1 ? ihi[t] : a1;
      for (int64_t i = lo; i <= hi; ++i) {
        double x = grid_nu(nu_min, dnu, i, wl_unit) - nu[t];
        sigma[i - i0] += I[t] * prof_point(kind, x, dnu, alpha[t], gamma[t]);
      }
    }
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Adjoint of L = sum_i w_i sigma_i (no counterpart in the paper).
 * Per kept line l, with f_li = f_l(nu_i - nu_l):
 *   G_l = sum_i w_i f_li,  Da_l = sum_i w_i df/dalpha,  Dg_l = sum_i w_i df/dgamma
 * and the absolute sums (|w| in place of w) that set the scale of each.
 *   dL/dA_l        = (I_l / A_l) G_l
 *   dL/dgamma_ref_l = I_l (T_ref/T)^n P Dg_l
 *   dL/dP          = sum_l I_l (gamma_l / P) Dg_l
 *   dL/dT (LTE) or dL/dT_rot (2T)
 *                  = sum_l I_l [ dlnI/dT G_l + (alpha_l / 2T) Da_l - (n_l gamma_l / T) Dg_l ]
 *   dL/dT_vib      = sum_l I_l dlnI/dT_vib G_l
 * with
 *   LTE: dlnI/dT = c2 E''/T^2 - (c2 nu/T^2) e^{-c2 nu/T}/(1 - e^{-c2 nu/T}) - Q'/Q
 *   2T : dlnI/dT_rot = c2 E''_rot/T_rot^2 - (c2 nu_rot/T_rot^2) e^{-X}/(1-e^{-X}) - Q_rot'/Q
 *        dlnI/dT_vib = c2 E''_vib/T_vib^2 - (c2 nu_vib/T_vib^2) e^{-X}/(1-e^{-X}) - Q_vib'/Q
 *        X = c2 (nu_vib/T_vib + nu_rot/T_rot).
 * (For the Gaussian-HWHM profile alpha does not depend on T.)
 * scal[0..2] = dL/dT, dL/dT_vib, dL/dP; scal[3..5] = the same with absolute values.
 * ------------------------------------------------------------------------ */

int orc_cross_section_grad(int kind, const double* E, const double* E_vib,
                           const int32_t* upper, const int32_t* lower, const void* A, int A_f32,
                           const double* nu, const double* I, const double* alpha, const double* gamma,
                           const float* n_T, const uint8_t* keep, const int64_t* ilo, const int64_t* ihi,
                           int64_t n, double T, double T_vib, double P, double T_ref, const double* Qd,
                           double nu_min, double dnu, const double* w,
                           double* dA, double* dgref, double* G, double* Gabs, double* scal) {
  if (kind & ORC_BINNED || kind >= ORC_PV_THOMPSON) return ORC_ERR_ARG;  /* sampled W-based profiles only */
  const double c2 = orc_c2();
  double* cT = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* cTv = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* cP = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* aT = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* aTv = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* aP = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < n; ++t) {
    dA[t] = 0.0; dgref[t] = 0.0; G[3 * t] = G[3 * t + 1] = G[3 * t + 2] = 0.0;
    Gabs[3 * t] = Gabs[3 * t + 1] = Gabs[3 * t + 2] = 0.0;
    if (!keep[t]) continue;
    double g0 = 0, ga = 0, gg = 0, h0 = 0, ha = 0, hg = 0;
    for (int64_t i = ilo[t]; i <= ihi[t]; ++i) {
      double x = (nu_min + (double)i * dnu) - nu[t];
      double f, fa, fg;
      prof_eval(kind, x, alpha[t], gamma[t], &f, &fa, &fg);
      g0 += w[i] * f; ga += w[i] * fa; gg += w[i] * fg;
      h0 += fabs(w[i] * f); ha += fabs(w[i] * fa); hg += fabs(w[i] * fg);
    }
    G[3 * t] = g0; G[3 * t + 1] = ga; G[3 * t + 2] = gg;
    Gabs[3 * t] = h0; Gabs[3 * t + 1] = ha; Gabs[3 * t + 2] = hg;
    double a = A_f32 ? (double)((const float*)A)[t] : ((const double*)A)[t];
    double Il = I[t];
    dA[t] = Il / a * g0;
    double dgam_dgref = (kind == ORC_LORENTZ || kind == ORC_VOIGT) ? pow(T_ref / T, (double)n_T[t]) * P : 0.0;
    dgref[t] = Il * dgam_dgref * gg;
    int64_t u = upper[t], l = lower[t];
    double dlnT, dlnTv = 0.0;
    if (T_vib > 0.0) {
      double ev_l = E_vib[l], er_l = E[l] - ev_l, ev_u = E_vib[u], er_u = E[u] - ev_u;
      double nv = ev_u - ev_l, nr = er_u - er_l;
      double X = c2 * (nv / T_vib + nr / T);
      double st = exp(-X) / (1.0 - exp(-X));
      dlnT = c2 * er_l / (T * T) - c2 * nr / (T * T) * st - Qd[1] / Qd[0];
      dlnTv = c2 * ev_l / (T_vib * T_vib) - c2 * nv / (T_vib * T_vib) * st - Qd[2] / Qd[0];
    } else {
      double X = c2 * nu[t] / T;
      double st = exp(-X) / (1.0 - exp(-X));
      dlnT = c2 * E[l] / (T * T) - c2 * nu[t] / (T * T) * st - Qd[1] / Qd[0];
    }
    double dalpha_dT = (kind == ORC_GAUSS_DOPPLER || kind == ORC_VOIGT) ? alpha[t] / (2.0 * T) : 0.0;
    double dgamma_dT = (kind == ORC_LORENTZ || kind == ORC_VOIGT) ? -(double)n_T[t] * gamma[t] / T : 0.0;
    double dgamma_dP = (kind == ORC_LORENTZ || kind == ORC_VOIGT) ? gamma[t] / P : 0.0;
    cT[t] = Il * (dlnT * g0 + dalpha_dT * ga + dgamma_dT * gg);
    cTv[t] = Il * dlnTv * g0;
    cP[t] = Il * dgamma_dP * gg;
    aT[t] = Il * (fabs(dlnT) * h0 + fabs(dalpha_dT) * ha + fabs(dgamma_dT) * hg);
    aTv[t] = Il * fabs(dlnTv) * h0;
    aP[t] = Il * fabs(dgamma_dP) * hg;
  }
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t t = 0; t < n; ++t) {
    s[0] += cT[t]; s[1] += cTv[t]; s[2] += cP[t];
    s[3] += aT[t]; s[4] += aTv[t]; s[5] += aP[t];
  }
  for (int j = 0; j < 6; ++j) scal[j] = s[j];
  free(cT); free(cTv); free(cP); free(aT); free(aTv); free(aP);
  return ORC_OK;
}
