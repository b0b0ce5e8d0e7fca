// Internal declarations of the pxc CUDA library (sm_103a).  Not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pxc.h"

namespace pxc {

// ---------------------------------------------------------------- constants (cgs, CODATA 2018 exact)
constexpr double kH = 6.62607015e-27;    // erg s
constexpr double kC = 2.99792458e10;     // cm/s
constexpr double kKB = 1.380649e-16;     // erg/K
constexpr double kNA = 6.02214076e23;    // 1/mol
constexpr double kPi = 3.14159265358979323846;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kExpMax = 709.78;       // largest Boltzmann exponent accepted
constexpr float kInvSqrtPi = 0.56418958354775628695f;
constexpr float kInvPi = 0.31830988618379067154f;
constexpr float kSqrtLn2 = 0.83255461115769775635f;
constexpr float kLog2e = 1.44269504088896340736f;

// Error bits latched in the workspace error word.
enum : unsigned {
  ERRB_ID = 1u << PXC_ERR_ID_RANGE,
  ERRB_NONFINITE = 1u << PXC_ERR_NONFINITE,
  ERRB_OVERFLOW = 1u << PXC_ERR_OVERFLOW,
  ERRB_TIMEOUT = 1u << PXC_ERR_TIMEOUT,
};

constexpr uint64_t kSentinelKey = ~0ull;  // sorts after every positive double

// ---------------------------------------------------------------- launch geometry
constexpr int kLinesPerBlockI = 2048;     // lines per CTA in the intensity pass (256 x 8)
constexpr int kThreadsI = 256;
constexpr int kUnitLines = 2048;         // lines per warp unit in the compacting intensity pass
#ifndef PXC_SORT_TILE
#define PXC_SORT_TILE 2048
#endif
// keys per CTA tile in a radix pass (256 threads x 8: 64 registers, four CTAs per SM; tiles of
// 4096 keys took 100 registers and measured 0.3 ms slower per 1e9-line step)
constexpr int kSortTile = PXC_SORT_TILE;
constexpr int kSortThreads = 256;
constexpr int kSortItems = kSortTile / kSortThreads;
constexpr int kQBlocks = 1184;            // 148 SMs x 8, fixed so the Q reduction order is fixed
constexpr int kThreadsQ = 256;

// Profile kernel tiles: segment widths are a runtime choice among the compiled configurations
// (see kernels_profile.cu); the workspace is sized for the narrowest and the widest.
constexpr int kNumTiles = 4;
constexpr int kBatchedDefaultTile = 0;  // 128-point segments (each temperature's non-zero lines only)
constexpr int kNumKinds = 11;
// Profile kinds (pxc_profile): sampled 0..3, binned 4..7, pseudo-Voigt 8..10.
__host__ __device__ constexpr bool is_binned(int kind) { return kind >= 4 && kind <= 7; }
__host__ __device__ constexpr bool is_pseudo_voigt(int kind) { return kind >= 8 && kind <= 10; }
constexpr long long kDefaultWaitLimit = 4000000000ll;  // ~2 s of clock cycles             // sampled and binned profile kinds (pxc_profile)
constexpr int kSegMin = 128;
constexpr int kSegMax = 2048;
constexpr int kStageLines = 256;          // lines per TMA stage (two per thread for the constants)
constexpr int kStages = 2;
constexpr int kItemLines = 32768;         // a segment with more lines is split into several items
constexpr int kPad = kStageLines + 8;     // padding of the per-line arrays so stages never read past them

// ---------------------------------------------------------------- per-condition constants
struct CondDev {
  double T, T_vib, P;
  float alpha_coef;     // Doppler HWHM / nu  (=(1/c) sqrt(2 N_A k_B T ln2 / M)), or 0
  float hwhm;           // fixed Gaussian HWHM
  float log2_tratio;    // log2(T_ref / T)
  float P_f;
  int32_t slot;         // intensity slot (distinct temperature pair)
  int32_t kind;
};

// Per-state record of the intensity pass, one 32-byte sector: E exact, the FP64 Boltzmann factor,
// g in FP64 and FP32 (no conversion per line), and log2 of the Boltzmann factor in FP32 (for the
// rejection bound).
struct __align__(32) StateFast {
  double E;
  double b;
  double g;
  float gf;
  float lb;
};

// Work item of the profile kernel: lines [begin, end) of the sorted list onto
// segment `seg` for condition `cond`; slot < 0 writes sigma directly, else a partial row.
struct Item {
  int32_t cond, seg, begin, end, slot, first_of_seg, n_of_seg, pad;
};

}  // namespace pxc

// ---------------------------------------------------------------- workspace (host struct)
struct pxc_workspace {
  pxc_capacity cap;
  char* base;
  size_t bytes;
  int accumulate;
  int sm_count;
  // cache of the Boltzmann table when accumulating chunks
  const double* cache_E;
  int64_t cache_n;
  double cache_T, cache_Tv;
  int cache_valid;
  // device regions
  unsigned* err;                 // error word
  unsigned long long* counters;  // [16]: queue, n_items, n_kept, stats...
  double* qpart;                 // [kQBlocks][max_cond][3]
  double* qres;                  // [max_cond][4]: Q, dQ, dQv, 1/(8 pi c Q)
  double2* srec;                 // [max_slots][max_states] {E, b}
  uint64_t* key;                 // [max_lines]
  double* Iv;                    // [max_lines] FP64 intensity (plain mode, by transition index)
  uint32_t* bcount;              // [nblk_I + 1]
  uint64_t* skey[2];             // sort ping-pong
  uint32_t* sidx[2];
  uint32_t* rcount;              // [256 * nblk_sort + 1]
  int4* pos;                     // [max_lines + pad] {ic, f bits, ilo, ihi}
  float2* par;                   // [max_lines + pad] {gamma_ref, n_T}
  float* Is;                     // [max_slots][max_lines + pad]
  int32_t* su;                   // sorted upper / lower / A (batched intensities)
  int32_t* sl;
  double* sA;
  double* sI;                    // [max_lines] per-slot FP64 intensity scratch
  int32_t* segr;                 // [2][max_seg]
  pxc::Item* items;              // [max_items]
  int32_t* seg_items;            // [max_cond * max_seg + 1] exclusive prefix of items
  float* partial;                // partial rows of the segment width in use
  pxc::CondDev* cond;            // [max_cond]
  int32_t* kexp;                 // [max_slots] exponent per slot
  unsigned long long* maxbits;   // [max_slots]
  int64_t max_seg, max_items, max_slots, nblk_I, nblk_sort;
  // host mirror of the last call
  int64_t last_nseg;
  int32_t last_nc;
  void* extra;                   // host-side bookkeeping of the ABI layer
};
