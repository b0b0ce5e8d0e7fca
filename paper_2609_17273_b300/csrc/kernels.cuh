// Kernel launchers of the pxc library (host functions, internal).
#pragma once
#include "pxc_internal.cuh"

namespace pxc {

// Slots of the workspace's u64 counter block: work-queue head, items, kept lines, lines with
// non-zero scaled intensity, window evaluations (all / non-zero lines), line-segment pairs, raw
// item total; CNT_N slots in all.
enum { CNT_QUEUE = 0, CNT_ITEMS = 1, CNT_KEPT = 2, CNT_NONZERO = 3, CNT_EVALS = 4, CNT_EVALS_NZ = 5, CNT_ALL = 6,
       CNT_ITEMS_RAW = 7, CNT_SLOT_NZ = 8, CNT_N = 16 };


// Host-side argument checks and per-condition constants shared by every entry point
// (pxc_api.cu); on failure they set the thread-local message and return the status.
struct SlotP;
pxc_status validate_states(const pxc_states* st);
pxc_status validate_condition(const pxc_condition& c, const pxc_states* st);
void set_last_error(const char* msg);

// Kernel launches issued by the library since load (all workspaces, all threads).
void note_launches(int n);
int64_t launches_total();

// Exact window / position arithmetic parameters (IEEE double, no contraction).
struct GridP {
  double nu_min, dnu, cut;        // on a wavelength grid nu_min, dnu hold lambda_min, dlambda
  int64_t n;
  double nu_keep_lo, nu_keep_hi;  // nu in [lo, hi] <=> window meets the grid (when exact_bounds)
  int exact_bounds;               // 0: evaluate the window per line
  double wl_unit;                 // 0: wavenumber grid; U > 0: wavelength grid with nu = U / lambda
  double nu_span_lo, nu_span_hi;  // every kept line has nu in [lo, hi] (the state-code prefilter)
  double inv_dnu;                 // 1 / dnu rounded to FP64 (a first guess of the window quotients)
};

struct SlotP {                    // one temperature pair
  double c2_T;                    // c2 / T   (T_rot for two-temperature)
  double c2_Tv;                   // c2 / T_vib, 0 for LTE
  double T, T_vib;                // T (T_rot) and T_vib (0 for LTE)
};
SlotP slot_constants(const pxc_condition& c);

// Partial sums per (block, slot): Q, and the moments for dQ/dT, dQ/dT_vib and the cooling function.
constexpr int kQMoments = 4;
void launch_boltzmann(const pxc_states* st, const SlotP* slots_dev, int nslot, double2* srec, int64_t srec_stride,
                      StateFast* sfast, double* qpart, double* qres, unsigned* err, cudaStream_t s,
                      const double* Ssum = nullptr, double* W_out = nullptr);

// Per-state 12-bit energy codes for the intensity pass's prefilter: q = floor((E - Emin) inv_res)
// for finite E (q <= kCodeMax), kCodeNone otherwise.  For every finite E, Emin + (q - 1) / inv_res
// <= E <= Emin + (q + 2) / inv_res, so nu = E_u - E_l lies within (q_u - q_l -+ 3) / inv_res.
// Five codes share one 64-bit word (state 5w + i at bits 12i .. 12i + 11; 80 MB for 5e7 states), so
// one 8-byte load fetches a code: the pass is limited by the L1 sectors of its random gathers, and
// a layout with codes across byte boundaries (three bytes per two states, 75 MB) needed two loads
// per code.  The random gathers find the table in L2 far more often than the 100 MB of 16-bit
// codes (measured 0.9 against 1.45 ms per 1e8 lines of gathers), for ~6 % candidates instead of
// ~3 %.  (8-bit codes, small enough for one die's L2 half, send ~40 % of the lines to the full test.)
using code_t = uint64_t;
constexpr int kCodeNone = 4095;
constexpr int kCodeMax = kCodeNone - 1;
inline size_t code_bytes(int64_t n_states) { return (size_t)((n_states + 4) / 5) * 8; }
struct QuantHdr {
  double Emin, inv_res;
  float res_f;      // 1 / inv_res rounded up
  float Emin_f;     // Emin rounded down
  float log2_gmax;  // log2 of the largest g, rounded up
  int enabled;      // 0: no finite energy range (prefilter off)
};
// Three reduction words (ordered keys of -Emin and Emax, max g) followed by the header.
constexpr int kQuantWords = 4;
void launch_cool_rates(const pxc_transitions* tr, const pxc_states* st, double* S, unsigned* err, cudaStream_t s);
void launch_state_codes(const pxc_states* st, code_t* code, unsigned long long* words, cudaStream_t s);

// How a line's value is formed from the per-state population factors b (value = num / den):
//   IMODE_ABS          absorption, LTE or two temperatures: g' A (b_l - b_u) / (8 pi c Q nu^2)
//                      (Eqs. abs intensity lte, nlte ab 2T)
//   IMODE_ABS_DENSITY  absorption, vibronic densities: g' A b_l (1 - exp(-c2 nu / T_rot)) /
//                      (8 pi c Q nu^2) (Eq. nlte ab pop density)
//   IMODE_EMISSION     emission, any population model: g' h c A nu b_u / (4 pi Q)
//                      (Eqs. ems intensity lte, nlte em 2T, nlte em pop density)
// invQ is 1/(8 pi c Q); h c / (4 pi Q) = 2 h c^2 invQ.
enum { IMODE_ABS = 0, IMODE_ABS_DENSITY = 1, IMODE_EMISSION = 2 };
constexpr double kTwoHC2 = 2.0 * kH * kC * kC;

__device__ __forceinline__ void line_value(int mode, double c2_T, double g, double A, double invQ, double bl,
                                           double bu, double nu, double* num, double* den) {
  if (mode == IMODE_EMISSION) {
    *num = g * A * invQ * (kTwoHC2 * bu * nu);
    *den = 1.0;
  } else if (mode == IMODE_ABS_DENSITY) {
    *num = g * A * invQ * (bl * -expm1(-c2_T * nu));
    *den = nu * nu;
  } else {
    *num = g * A * invQ * (bl - bu);
    *den = nu * nu;
  }
}

struct BoundP {
  float log2_thr;
  float log2_invQ;
  float c2_T;
  int lte;
  int mode;      // IMODE_*
  double c2_Td;  // c2 / T (T_rot), FP64
};
// Intensity pass of the cross-section path: prefilter (candidates per unit into cand_* / ccount,
// which need max_lines entries and one count per unit) and exact selection (kept lines staged per
// unit into kstage / istage, counts into ucount, FP64 intensities by transition index into Iv).
void launch_lines_compact(const pxc_transitions* tr, int64_t ns, const code_t* code, const QuantHdr* qh,
                          const StateFast* sfast,
                          const double* qres, const GridP& gp, double threshold, const BoundP& bp, int with_I,
                          uint32_t* cand_t, uint64_t* cand_ul, uint64_t* cand_a, uint32_t* ccount,
                          uint64_t* kstage, uint32_t* istage, double* Iv, uint32_t* ucount, int64_t nunit,
                          unsigned long long* maxbits, unsigned* err, cudaStream_t s);
void launch_compact_staged(const uint64_t* kstage, const uint32_t* istage, const uint32_t* uoff, int64_t nunit,
                           uint64_t* okey, uint32_t* oidx, cudaStream_t s);

void launch_lines(const pxc_transitions* tr, const int32_t* g, int64_t ns, const double2* srec,
                  const double* qres, const GridP& gp, const BoundP& bp, int use_grid, double threshold,
                  int with_intensity,
                  uint64_t* key, double* Iv, double* nu_out, uint32_t* bcount, int64_t nblk,
                  unsigned long long* maxbits, unsigned* err, cudaStream_t s);

void launch_scan_counts(uint32_t* bcount, int64_t nblk, unsigned long long* total, cudaStream_t s);


// Sorts (key, idx) pairs of device count *n_dev (<= n_max) by key, stable.  Result
// ends in buffer 0 (8 passes).
void launch_radix_sort(uint64_t* key[2], uint32_t* idx[2], const unsigned long long* n_dev, int64_t n_max,
                       uint32_t* rcount, cudaStream_t s);

void launch_exponent(const unsigned long long* maxbits, int32_t* kexp, int32_t* sigma_exp_inout,
                     int accumulate, float* sigma, int64_t n_grid, cudaStream_t s);

void launch_prepare(const uint64_t* skey, const uint32_t* sidx, const unsigned long long* n_dev, int64_t n_max,
                    const GridP& gp, const float* gamma_ref, const float* n_T, const double* Iv,
                    const int32_t* kexp, int4* pos, float2* par, float* Is,
                    const pxc_transitions* gather_tr, int32_t* su, int32_t* sl, double* sA,
                    int64_t* perm_out, unsigned long long* counters, cudaStream_t s);

void launch_sorted_intensity(const int32_t* su, const int32_t* sl, const double* sA, const unsigned long long* n_dev,
                             int64_t n_max, const int32_t* g, const double2* srec, const double* qres,
                             const BoundP& bp, double threshold, double* sI, unsigned long long* maxbits,
                             cudaStream_t s);

void launch_scale(const double* sI, const unsigned long long* n_dev, int64_t n_max, const int32_t* kexp,
                  float* Is, unsigned long long* counters, cudaStream_t s);

void launch_segments(const int4* pos, const unsigned long long* n_dev, int64_t nseg, int seg, int32_t* segr,
                     cudaStream_t s);

// cond_list: the condition of each group of nseg items (n_c entries), or null for 0 .. n_c-1.
void launch_items(const int32_t* segr, int64_t nseg, int n_c, int item_lines, int32_t* seg_items,
                  Item* items, unsigned long long* counters, int64_t max_items, int64_t target_items,
                  int64_t max_partial, const int32_t* cond_list, cudaStream_t s);
// Stable compaction of the first *n_dev sorted lines with non-zero scaled intensity Is into
// pos_c / par_c / Is_c (count to *nnz_dev); bcount needs n_max / kUnitLines + 2 entries.
void launch_compact_nonzero(const int4* pos, const float2* par, const float* Is, const unsigned long long* n_dev,
                            int64_t n_max, uint32_t* bcount, unsigned long long* nnz_dev, int4* pos_c, float2* par_c,
                            float* Is_c, cudaStream_t s);

// Adds each (condition, segment) group's partial rows to its sigma row (cond_list as in launch_items).
void launch_reduce_partials(const Item* items, const int32_t* seg_items, int64_t nseg, int seg, int n_c,
                            const float* partial, float* sigma, int64_t n_grid, const int32_t* cond_list,
                            cudaStream_t s);

void launch_stick_out(const double* Iv, const uint64_t* key, int64_t n, const int32_t* kexp, float* I_scaled,
                      cudaStream_t s);

// Profile kernels (kernels_profile.cu).
struct ProfP {
  const int4* pos;
  const float2* par;
  const float* Is;
  int64_t is_stride;       // floats between intensity slots
  const CondDev* cond;
  const Item* items;
  const unsigned long long* n_items;
  unsigned long long* queue;
  float* sigma;            // [n_c][n_grid]
  float* partial;          // partial rows of the segment width in use
  int64_t n_grid;
  double nu_min, dnu;
  int accumulate;
  int kind;
  unsigned* err;
  long long spin_limit;   // bound of the waits for staged records (clock cycles)
  long long drain_limit;  // bound of the final wait for copies still in flight after a timeout
  double wl_unit;         // > 0: wavelength grid (nu_min, dnu hold lambda_min, dlambda)
};
void launch_profile(const ProfP& p, int tile, int grid_ctas, cudaStream_t s);
// Profile accumulation on a wavelength grid: 128-point segments, one work item per CTA.
constexpr int kSegWl = 128;
void launch_profile_wl(const ProfP& p, int64_t max_items, cudaStream_t s);
int profile_occupancy(int kind, int tile);
int tile_seg(int tile);

struct AdjP {
  const int4* pos;
  const float2* par;
  const float* Is;
  const uint32_t* sidx;    // sorted position -> transition index
  const int32_t* su;       // sorted upper / lower ids
  const int32_t* sl;
  const double* sA;
  const double2* srec;     // {E, b} of the condition's slot
  const double* E_vib;
  const float* n_T;        // per transition
  const double* qres;      // Q, dQ, dQv
  const float* w;          // dL/dsigma_s [n_grid]
  const unsigned long long* n_dev;
  int64_t n_max;
  int64_t n_grid;
  double nu_min, dnu, T, T_vib, P, T_ref, c2;
  CondDev cond;
  int kind;
  float* dA;               // [n_trans] by transition index
  float* dgref;
  double* lineT;           // [n_max] per-line contributions (sorted order) to the scalars
  double* lineTv;
  double* lineP;
};
void launch_adjoint(const AdjP& p, cudaStream_t s);
// Fixed-order FP64 sums of the per-line shares; `scratch` holds adjoint_reduce_scratch_bytes().
size_t adjoint_reduce_scratch_bytes();
void launch_adjoint_reduce(const double* lineT, const double* lineTv, const double* lineP,
                           const unsigned long long* n_dev, double* scratch, double* outT, double* outTv,
                           double* outP, cudaStream_t s);

}  // namespace pxc
