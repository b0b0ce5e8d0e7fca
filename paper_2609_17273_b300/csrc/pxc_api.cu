// C ABI of the pxc library: argument checks, workspace carving, orchestration
// of the kernels on the caller's stream, and the chunked host-streaming loop.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kernels.cuh"

using namespace pxc;

namespace {

thread_local char g_msg[512] = "";

pxc_status fail(pxc_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return st;
}

pxc_status cuda_check(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PXC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return PXC_OK;
}


constexpr int kWinCap = 16384;  // largest cut-off window (points) the item tables are sized for

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t err, counters, qpart, qres, slots, cond, srec, sfast, key, Iv, bcount, skey0, skey1, sidx0, sidx1, rcount, pos,
      par, Is, su, sl, sA, sI, segr, seg_items, items, partial, kexp, maxbits, params, code, qwords, pos_c, par_c,
      Is_c, condlist, total;
  int64_t max_seg, max_items, max_slots, nblk_I, nblk_sort, max_cond, is_stride;
  int64_t partial_floats;  // partial-row buffer; a tile of S points has partial_floats / S rows
};

// Largest number of partial rows a split single-condition call can need with segments of
// `seg` points: every line meets at most kWinCap / seg + 2 segments, and items hold at
// least kItemLines lines unless the row budget allows more splitting.
int64_t split_rows(int64_t ml, int seg) { return ml * (kWinCap / seg + 2) / kItemLines + 1; }

Layout make_layout(const pxc_capacity& c) {
  Layout L{};
  const int64_t ml = std::max<int64_t>(c.max_lines, 1);
  L.max_cond = std::max<int32_t>(c.max_conditions, 1);
  L.max_slots = c.max_temperatures > 0 ? std::min<int64_t>(c.max_temperatures, L.max_cond) : L.max_cond;
  L.max_seg = (std::max<int64_t>(c.max_grid, 1) + kSegMin - 1) / kSegMin;  // narrowest tile: most segments
  L.nblk_I = (ml + kLinesPerBlockI - 1) / kLinesPerBlockI;
  L.nblk_sort = (ml + kSortTile - 1) / kSortTile;
  L.partial_floats = 0;
  for (int t = 0; t < kNumTiles; ++t)
    L.partial_floats = std::max<int64_t>(L.partial_floats, split_rows(ml, tile_seg(t)) * tile_seg(t));
  // one item per (condition, segment) plus the split items, whose partial rows the partial-row
  // buffer bounds (batched calls split too)
  L.max_items = L.max_cond * L.max_seg + L.partial_floats / kSegMin;
  L.is_stride = ((ml + kPad) + 3) & ~(int64_t)3;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
  L.err = take(256);
  L.counters = take(CNT_N * 8);
  L.qpart = take((size_t)kQBlocks * L.max_cond * kQMoments * 8);
  L.qres = take((size_t)L.max_cond * 4 * 8);
  L.slots = take((size_t)L.max_cond * sizeof(SlotP));
  L.cond = take((size_t)L.max_cond * sizeof(CondDev));
  L.srec = take((size_t)std::max<int64_t>(c.max_states, 1) * 16);
  L.sfast = take((size_t)std::max<int64_t>(c.max_states, 1) * sizeof(StateFast));
  L.key = take((size_t)ml * 8);
  L.Iv = take((size_t)ml * 8);
  L.bcount = take((size_t)((ml + kUnitLines - 1) / kUnitLines + 1) * 4);  // per unit (>= per block)
  L.skey0 = take((size_t)ml * 8);
  L.skey1 = take((size_t)ml * 8);
  L.sidx0 = take((size_t)ml * 4);
  L.sidx1 = take((size_t)ml * 4);
  L.rcount = take((size_t)(256 * L.nblk_sort + 256) * 4);
  L.pos = take((size_t)(ml + kPad) * 16);
  L.par = take((size_t)(ml + kPad) * 8);
  L.Is = take((size_t)L.max_slots * L.is_stride * 4);
  L.su = take((size_t)ml * 4);
  L.sl = take((size_t)ml * 4);
  L.sA = take((size_t)ml * 8);
  L.sI = take((size_t)ml * 8);
  L.segr = take((size_t)2 * L.max_seg * 4);
  L.seg_items = take((size_t)(L.max_cond * L.max_seg + 1) * 4);
  L.items = take((size_t)L.max_items * sizeof(Item));
  L.partial = take((size_t)L.partial_floats * 4);
  L.kexp = take((size_t)L.max_slots * 2 * 4);
  L.maxbits = take((size_t)L.max_slots * 8);
  L.params = take(4096);
  L.code = take(code_bytes(std::max<int64_t>(c.max_states, 1)));
  L.qwords = take(kQuantWords * 8 + sizeof(QuantHdr));
  // batched calls: the lines of one temperature with non-zero scaled intensity, and the
  // conditions grouped by temperature
  const size_t nzl = L.max_cond > 1 ? (size_t)(ml + kPad) : 0;
  L.pos_c = take(nzl * 16);
  L.par_c = take(nzl * 8);
  L.Is_c = take(nzl * 4);
  L.condlist = take((size_t)L.max_cond * 4);
  L.total = o;
  return L;
}

bool bad_ptr(const void* p) { return p == nullptr; }

pxc_status check_states(const pxc_states* st) {
  if (!st || st->n < 0 || (st->n > 0 && (bad_ptr(st->E) || bad_ptr(st->g))))
    return fail(PXC_ERR_ARG, "states: null pointer or n < 0");
  if (st->n > INT32_MAX) return fail(PXC_ERR_ARG, "states: more than 2^31-1 states");
  return PXC_OK;
}

pxc_status check_trans(const pxc_transitions* tr) {
  if (!tr || tr->n < 0 || (tr->n > 0 && (bad_ptr(tr->upper) || bad_ptr(tr->lower) || bad_ptr(tr->A))))
    return fail(PXC_ERR_ARG, "transitions: null pointer or n < 0");
  return PXC_OK;
}

pxc_status check_cond(const pxc_condition& c, bool need_vib, const pxc_states* st) {
  if (!(c.T > 0.0) || !std::isfinite(c.T)) return fail(PXC_ERR_ARG, "condition: T must be > 0");
  if (!std::isfinite(c.T_vib)) return fail(PXC_ERR_ARG, "condition: T_vib not finite");
  if (c.T_vib > 0.0 && (!st || bad_ptr(st->E_vib))) return fail(PXC_ERR_ARG, "condition: T_vib > 0 needs E_vib");
  if (st && st->n_vib && bad_ptr(st->E_vib)) return fail(PXC_ERR_ARG, "states: vibronic densities need E_vib");
  if (st && st->n_vib && c.T_vib > 0.0)
    return fail(PXC_ERR_ARG, "condition: T_vib > 0 with vibronic densities is ambiguous");
  (void)need_vib;
  return PXC_OK;
}

pxc_status check_grid(const pxc_grid* g, double cut) {
  if (!g || !(g->dnu > 0.0) || g->n < 1 || !std::isfinite(g->nu_min) || !std::isfinite(g->dnu))
    return fail(PXC_ERR_ARG, "grid: dnu must be > 0 and n >= 1");
  if (!(g->wl_unit >= 0.0) || !std::isfinite(g->wl_unit))
    return fail(PXC_ERR_ARG, "grid: wl_unit must be 0 (wavenumbers) or > 0 (wavelengths)");
  if (g->wl_unit > 0.0 && !(g->nu_min > 0.0)) return fail(PXC_ERR_ARG, "grid: wavelengths must be > 0");
  if (!(cut >= 0.0) || !std::isfinite(cut)) return fail(PXC_ERR_ARG, "cutoff must be finite and >= 0");
  if (g->n > (int64_t)INT32_MAX - 2 * kSegMax) return fail(PXC_ERR_ARG, "grid: too many points");
  return PXC_OK;
}

// Host replicas of the window arithmetic (plain IEEE double; nvcc passes -ffp-contract=off to the host compiler).
double win_hi_idx(double nu, double cut, double nu_min, double dnu) { return std::floor(((nu + cut) - nu_min) / dnu); }
double win_lo_idx(double nu, double cut, double nu_min, double dnu) { return std::ceil(((nu - cut) - nu_min) / dnu); }

uint64_t dbits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
double bitsd(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }

// Exact bounds on nu (positive doubles) such that the window meets the grid: both
// predicates are monotone in nu, so bisection over the ordered bit patterns of
// positive doubles finds the smallest nu with i_hi >= 0 and the largest with i_lo <= n-1.
GridP make_gridp(const pxc_grid& g, double cut) {
  GridP gp{};
  gp.nu_min = g.nu_min; gp.dnu = g.dnu; gp.cut = cut; gp.n = g.n;
  gp.inv_dnu = 1.0 / g.dnu;
  gp.wl_unit = g.wl_unit;
  gp.exact_bounds = 0;
  const double last = g.nu_min + (double)(g.n - 1) * g.dnu;
  if (g.wl_unit > 0.0) {
    // wavelength grid: kept lines have nu within [U/lambda_max - cut, U/lambda_min + cut]
    // (widened by 1e-6 relative for the rounding of the window arithmetic); windows per line
    const double a = g.wl_unit / last - cut, b = g.wl_unit / g.nu_min + cut;
    gp.nu_span_lo = std::max(0.0, a - 1e-6 * std::fabs(a) - 1e-6 * cut);
    gp.nu_span_hi = b + 1e-6 * std::fabs(b);
    return gp;
  }
  gp.nu_span_lo = std::max(g.nu_min - cut, 0.0);
  gp.nu_span_hi = last + cut;
  if (!(cut >= 1.5 * g.dnu)) return gp;  // short windows can fall between points: test each line
  const uint64_t LO = 1, HI = dbits(1.7976931348623157e308);
  auto p_lo = [&](uint64_t b) { return win_hi_idx(bitsd(b), cut, g.nu_min, g.dnu) >= 0.0; };
  auto p_hi = [&](uint64_t b) { return win_lo_idx(bitsd(b), cut, g.nu_min, g.dnu) <= (double)(g.n - 1); };
  double lo, hi;
  if (p_lo(LO)) lo = bitsd(LO);
  else if (!p_lo(HI)) lo = INFINITY;
  else {
    uint64_t a = LO, b = HI;  // p(a) false, p(b) true
    while (b - a > 1) { uint64_t m = a + (b - a) / 2; if (p_lo(m)) b = m; else a = m; }
    lo = bitsd(b);
  }
  if (p_hi(HI)) hi = bitsd(HI);
  else if (!p_hi(LO)) hi = -INFINITY;
  else {
    uint64_t a = LO, b = HI;  // p(a) true, p(b) false
    while (b - a > 1) { uint64_t m = a + (b - a) / 2; if (p_hi(m)) a = m; else b = m; }
    hi = bitsd(a);
  }
  gp.nu_keep_lo = lo;
  gp.nu_keep_hi = hi;
  gp.exact_bounds = 1;
  return gp;
}

template <typename T>
T* at(pxc_workspace* ws, size_t off) { return reinterpret_cast<T*>(ws->base + off); }

// One captured pxc_cross_section: the call's key (every pointer and value it depends on), the
// instantiated graph, the kernels it holds and the host-side bookkeeping of the call.
struct GraphEntry {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec;
  int64_t kernels;
  int64_t last_nseg;
  int last_seg, last_tile, last_nc;
};
constexpr size_t kGraphCacheMax = 8;

struct WsExtra {
  Layout L;
  void* h_params;        // pinned host staging of small parameter blocks
  unsigned* h_err;
  unsigned long long* h_cnt;
  cudaStream_t copy_stream;
  cudaEvent_t ev_copied[2], ev_done[2];
  int occ[kNumKinds][kNumTiles];  // resident profile CTAs per SM for each kind and tile
  int emission;           // emission intensities instead of absorption
  long long wait_limit;   // bound of the profile kernel's waits for staged records (clock cycles)
  const double* cache_nvib;  // densities the cached Boltzmann table was built with
  int tile[kNumKinds][2];         // tile used for each kind, [single condition, batched]
  // last call
  int64_t last_nseg;
  int last_seg, last_tile;
  int64_t last_nkept_max;
  // optional CUDA-event timing of the passes: [0] intensity, [1] compaction+sort+prepare, [2] profile
  int timing;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_used;  // (pass, index of the start event)
  size_t ev_next;
  // CUDA-graph replay of pxc_cross_section (pxc_set_graphs)
  int graphs;
  int capturing;
  cudaStream_t cap_stream;
  std::vector<GraphEntry> gcache;  // most recently used last
  int64_t graph_hits, graph_captures;
  // pxc_set_reuse_forward: the arguments of the single-condition call whose kept, sorted line list
  // (with the per-line ids and A the adjoint needs) the workspace holds; empty when none
  int reuse_fwd;
  std::vector<unsigned char> fwd_key;
};

// Records a timing event for `pass` (start or end) when timing is on.
void tmark(pxc_workspace* ws, int pass, bool start, cudaStream_t s);

WsExtra* X(pxc_workspace* ws) { return reinterpret_cast<WsExtra*>(ws->extra); }

// Small parameter blocks reach device memory as kernel arguments (captured by value in
// CUDA graphs, no host staging whose lifetime would matter, no synchronisation).
struct ParamBlock {
  unsigned char b[12288];
};
__global__ void k_store_params(const __grid_constant__ ParamBlock blk, unsigned nbytes, unsigned char* dst) {
  for (unsigned i = threadIdx.x; i < nbytes; i += blockDim.x) dst[i] = blk.b[i];
}

pxc_status upload(pxc_workspace* ws, void* dev, const void* host, size_t bytes, cudaStream_t s) {
  (void)ws;
  const unsigned char* h = (const unsigned char*)host;
  for (size_t off = 0; off < bytes; off += sizeof(ParamBlock)) {
    ParamBlock blk;
    size_t n = std::min(sizeof(ParamBlock), bytes - off);
    memcpy(blk.b, h + off, n);
    k_store_params<<<1, 256, 0, s>>>(blk, (unsigned)n, (unsigned char*)dev + off);
    note_launches(1);
  }
  return cuda_check("parameter upload");
}

SlotP make_slot(const pxc_condition& c) {
  const double c2 = kH * kC / kKB;
  SlotP sp{};
  sp.c2_T = c2 / c.T;
  sp.c2_Tv = c.T_vib > 0.0 ? c2 / c.T_vib : 0.0;
  sp.T = c.T;
  sp.T_vib = c.T_vib > 0.0 ? c.T_vib : 0.0;
  return sp;
}

CondDev make_cond(const pxc_condition& c, const pxc_profile_args& pa, int slot) {
  CondDev cd{};
  cd.T = c.T; cd.T_vib = c.T_vib; cd.P = c.P;
  cd.alpha_coef = (float)(std::sqrt(2.0 * kNA * kKB * c.T * kLn2 / pa.mass_da) / kC);
  cd.hwhm = (float)pa.hwhm;
  cd.log2_tratio = (float)std::log2(pa.T_ref / c.T);
  cd.P_f = (float)c.P;
  cd.slot = slot;
  cd.kind = pa.kind;
  return cd;
}

// Width kind of a profile: binned kinds take the widths of their base kind, pseudo-Voigts those of
// the Voigt kind.
int width_kind(int kind) { return is_pseudo_voigt(kind) ? PXC_VOIGT : (kind & 3); }

pxc_status check_prof(const pxc_profile_args* pa, const pxc_transitions* tr) {
  if (!pa) return fail(PXC_ERR_ARG, "profile args: null");
  if (pa->kind < PXC_GAUSS_DOPPLER || pa->kind > PXC_PV_LIULIN) return fail(PXC_ERR_ARG, "profile: unknown kind");
  const int base = width_kind(pa->kind);
  if ((base == PXC_GAUSS_DOPPLER || base == PXC_VOIGT) && !(pa->mass_da > 0.0))
    return fail(PXC_ERR_ARG, "profile: mass must be > 0");
  if (base == PXC_GAUSS_HWHM && !(pa->hwhm > 0.0)) return fail(PXC_ERR_ARG, "profile: hwhm must be > 0");
  if ((base == PXC_LORENTZ || base == PXC_VOIGT) && tr->n > 0 && (bad_ptr(pa->gamma_ref) || bad_ptr(pa->n_T)))
    return fail(PXC_ERR_ARG, "profile: gamma_ref and n_T required");
  if ((base == PXC_LORENTZ || base == PXC_VOIGT) && !(pa->T_ref > 0.0))
    return fail(PXC_ERR_ARG, "profile: T_ref must be > 0");
  if (!(pa->cutoff >= 0.0)) return fail(PXC_ERR_ARG, "profile: cutoff must be >= 0");
  return PXC_OK;
}

// Runs K-Q for one slot into srec/qres[slot] unless cached (accumulate mode).
void run_boltzmann(pxc_workspace* ws, const pxc_states* st, const pxc_condition& c, int slot, cudaStream_t s,
                   bool allow_cache) {
  WsExtra* x = X(ws);
  if (allow_cache && ws->cache_valid && ws->cache_E == st->E && ws->cache_n == st->n && ws->cache_T == c.T &&
      ws->cache_Tv == c.T_vib && x->cache_nvib == st->n_vib)
    return;
  SlotP sp = make_slot(c);
  SlotP* dslot = at<SlotP>(ws, x->L.slots) + slot;
  upload(ws, dslot, &sp, sizeof sp, s);
  launch_boltzmann(st, dslot, 1, at<double2>(ws, x->L.srec), 0, at<StateFast>(ws, x->L.sfast),
                   at<double>(ws, x->L.qpart), at<double>(ws, x->L.qres) + 4 * slot, ws->err, s);
  // the energy codes depend on E only; rebuilt whenever the state table is
  if (slot == 0) launch_state_codes(st, at<code_t>(ws, x->L.code), at<unsigned long long>(ws, x->L.qwords), s);
  ws->cache_valid = allow_cache ? 1 : 0;
  ws->cache_E = st->E; ws->cache_n = st->n; ws->cache_T = c.T; ws->cache_Tv = c.T_vib;
  x->cache_nvib = st->n_vib;
}

const QuantHdr* qhdr(pxc_workspace* ws) {
  return reinterpret_cast<const QuantHdr*>(at<unsigned long long>(ws, X(ws)->L.qwords) + kQuantWords);
}

BoundP make_bound(pxc_workspace* ws, const pxc_states* st, const pxc_condition& c, double threshold) {
  BoundP bp{};
  bp.log2_thr = threshold > 0.0 ? (float)(std::log2(threshold) - 1e-3) : -INFINITY;
  bp.log2_invQ = 0.f;
  bp.lte = c.T_vib > 0.0 ? 0 : 1;
  bp.c2_Td = kH * kC / kKB / c.T;
  bp.c2_T = (float)bp.c2_Td;
  bp.mode = X(ws)->emission ? IMODE_EMISSION : (st->n_vib ? IMODE_ABS_DENSITY : IMODE_ABS);
  return bp;
}

// The intensity pass's candidate arrays reuse sort buffers that are free until the kept lines are
// compacted (sidx0, skey0, skey1) and the radix counts (one count per unit).
#define CAND_BUFFERS(ws, L)                                                                       \
  at<uint32_t>(ws, (L).sidx0), at<uint64_t>(ws, (L).skey0), at<uint64_t>(ws, (L).skey1), \
      at<uint32_t>(ws, (L).rcount)

// Lines -> kept, sorted, prepared (plain single-condition path).  with_gather fills su/sl/sA.
pxc_status front_plain(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr, const pxc_condition& c,
                       const GridP& gp, const pxc_profile_args* pa, double threshold, int32_t* sig_exp, float* sigma,
                       int64_t n_grid, bool with_gather, cudaStream_t s) {
  WsExtra* x = X(ws);
  const Layout& L = x->L;
  unsigned long long* cnt = at<unsigned long long>(ws, L.counters);
  run_boltzmann(ws, st, c, 0, s, ws->accumulate != 0);
  cudaMemsetAsync(at<unsigned long long>(ws, L.maxbits), 0, 8, s);
  const int64_t nunit = (tr->n + kUnitLines - 1) / kUnitLines;
  tmark(ws, 0, true, s);
  BoundP bp = make_bound(ws, st, c, threshold);
  launch_lines_compact(tr, st->n, at<code_t>(ws, L.code), qhdr(ws), at<StateFast>(ws, L.sfast),
                       at<double>(ws, L.qres), gp, threshold, bp, 1, CAND_BUFFERS(ws, L),
                       at<uint64_t>(ws, L.key), at<uint32_t>(ws, L.sidx1), at<double>(ws, L.Iv),
                       at<uint32_t>(ws, L.bcount), nunit, at<unsigned long long>(ws, L.maxbits), ws->err, s);
  tmark(ws, 0, false, s);
  tmark(ws, 1, true, s);
  if (nunit) launch_scan_counts(at<uint32_t>(ws, L.bcount), nunit, cnt + CNT_KEPT, s);
  launch_compact_staged(at<uint64_t>(ws, L.key), at<uint32_t>(ws, L.sidx1), at<uint32_t>(ws, L.bcount), nunit,
                        at<uint64_t>(ws, L.skey0), at<uint32_t>(ws, L.sidx0), s);
  uint64_t* keys[2] = {at<uint64_t>(ws, L.skey0), at<uint64_t>(ws, L.skey1)};
  uint32_t* idxs[2] = {at<uint32_t>(ws, L.sidx0), at<uint32_t>(ws, L.sidx1)};
  launch_radix_sort(keys, idxs, cnt + CNT_KEPT, tr->n, at<uint32_t>(ws, L.rcount), s);
  int32_t* kexp = at<int32_t>(ws, L.kexp);
  launch_exponent(at<unsigned long long>(ws, L.maxbits), kexp, sig_exp, ws->accumulate, sigma, n_grid, s);
  launch_prepare(keys[0], idxs[0], cnt + CNT_KEPT, tr->n, gp, pa ? pa->gamma_ref : nullptr, pa ? pa->n_T : nullptr,
                 at<double>(ws, L.Iv), kexp, at<int4>(ws, L.pos), at<float2>(ws, L.par), at<float>(ws, L.Is),
                 with_gather ? tr : nullptr, at<int32_t>(ws, L.su), at<int32_t>(ws, L.sl), at<double>(ws, L.sA),
                 nullptr, cnt, s);
  tmark(ws, 1, false, s);
  return cuda_check("line pipeline");
}

void tmark(pxc_workspace* ws, int pass, bool start, cudaStream_t s) {
  WsExtra* x = X(ws);
  if (!x->timing || x->capturing) return;
  if (x->ev_next + 1 >= x->ev_pool.size()) return;  // pool exhausted: stop recording
  cudaEvent_t e = x->ev_pool[x->ev_next];
  if (start) x->ev_used.push_back({pass, (int)x->ev_next});
  cudaEventRecord(e, s);
  ++x->ev_next;
}

int profile_ctas(pxc_workspace* ws, int kind, int tile) {
  WsExtra* x = X(ws);
  int occ = x->occ[kind][tile] > 0 ? x->occ[kind][tile] : 1;
  return ws->sm_count * occ;
}

}  // namespace

namespace pxc {
void set_last_error(const char* msg) { snprintf(g_msg, sizeof g_msg, "%s", msg); }
// The argument checks and per-condition constants of the workspace entry points, shared with
// the allocation-free partition function so that both accept exactly the same inputs.
pxc_status validate_states(const pxc_states* st) { return check_states(st); }
pxc_status validate_condition(const pxc_condition& c, const pxc_states* st) { return check_cond(c, false, st); }
SlotP slot_constants(const pxc_condition& c) { return make_slot(c); }
}  // namespace pxc

extern "C" {

const char* pxc_last_error(void) { return g_msg; }

int64_t pxc_kernel_launches(void) { return launches_total(); }

pxc_status pxc_workspace_query(const pxc_capacity* cap, size_t* bytes) {
  if (!cap || !bytes || cap->max_states < 0 || cap->max_lines < 0 || cap->max_grid < 0 || cap->max_conditions < 0)
    return fail(PXC_ERR_ARG, "workspace_query: bad capacity");
  if (cap->max_lines > (int64_t)INT32_MAX - 2 * kPad) return fail(PXC_ERR_ARG, "max_lines above 2^31");
  *bytes = make_layout(*cap).total;
  return PXC_OK;
}

pxc_status pxc_workspace_create(const pxc_capacity* cap, void* scratch, size_t bytes, pxc_workspace** out) {
  size_t need = 0;
  pxc_status st = pxc_workspace_query(cap, &need);
  if (st) return st;
  if (!out || !scratch || ((uintptr_t)scratch & 255)) return fail(PXC_ERR_ARG, "workspace_create: bad buffer");
  if (bytes < need) return fail(PXC_ERR_CAPACITY, "workspace_create: %zu bytes given, %zu needed", bytes, need);
  pxc_workspace* ws = (pxc_workspace*)calloc(1, sizeof(pxc_workspace));
  WsExtra* x = new WsExtra();
  if (!ws || !x) return fail(PXC_ERR_ARG, "out of host memory");
  x->L = make_layout(*cap);
  ws->cap = *cap;
  ws->base = (char*)scratch;
  ws->bytes = bytes;
  ws->extra = x;
  ws->err = at<unsigned>(ws, x->L.err);
  ws->counters = at<unsigned long long>(ws, x->L.counters);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ws->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (cudaHostAlloc(&x->h_params, 4096, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&x->h_err, 64, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&x->h_cnt, CNT_N * 8, cudaHostAllocDefault) != cudaSuccess)
    return fail(PXC_ERR_CUDA, "pinned host staging allocation failed");
  cudaStreamCreateWithFlags(&x->copy_stream, cudaStreamNonBlocking);
  for (int i = 0; i < 2; ++i) {
    cudaEventCreateWithFlags(&x->ev_copied[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&x->ev_done[i], cudaEventDisableTiming);
  }
  for (int k = 0; k < kNumKinds; ++k) {
    for (int t = 0; t < kNumTiles; ++t) x->occ[k][t] = profile_occupancy(k, t);
    // defaults: narrow segments balance dense spectra best, for single-condition calls and for
    // batched tables (which profile each temperature's non-zero lines only)
    x->tile[k][0] = 0;
    x->tile[k][1] = kBatchedDefaultTile;
  }
  x->wait_limit = kDefaultWaitLimit;
  cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking);
  cudaMemset(ws->err, 0, 256);
  cudaMemset(ws->counters, 0, CNT_N * 8);
  cudaDeviceSynchronize();
  *out = ws;
  return cuda_check("workspace_create");
}

pxc_status pxc_workspace_destroy(pxc_workspace* ws) {
  if (!ws) return PXC_OK;
  WsExtra* x = X(ws);
  cudaStreamSynchronize(x->copy_stream);
  cudaStreamDestroy(x->copy_stream);
  for (int i = 0; i < 2; ++i) { cudaEventDestroy(x->ev_copied[i]); cudaEventDestroy(x->ev_done[i]); }
  for (auto& e : x->ev_pool) cudaEventDestroy(e);
  for (auto& g : x->gcache) cudaGraphExecDestroy(g.exec);
  cudaStreamDestroy(x->cap_stream);
  cudaFreeHost(x->h_params);
  cudaFreeHost(x->h_err);
  cudaFreeHost(x->h_cnt);
  delete x;
  free(ws);
  return PXC_OK;
}

pxc_status pxc_set_wait_limit(pxc_workspace* ws, int64_t cycles) {
  if (!ws || cycles < 0) return fail(PXC_ERR_ARG, "set_wait_limit: null workspace or negative limit");
  X(ws)->wait_limit = cycles;
  return PXC_OK;
}

pxc_status pxc_set_emission(pxc_workspace* ws, int on) {
  if (!ws) return fail(PXC_ERR_ARG, "set_emission: null workspace");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  X(ws)->emission = on ? 1 : 0;
  return PXC_OK;
}

pxc_status pxc_set_accumulate(pxc_workspace* ws, int on) {
  if (!ws) return fail(PXC_ERR_ARG, "null workspace");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  ws->accumulate = on ? 1 : 0;
  if (!on) ws->cache_valid = 0;
  return PXC_OK;
}

pxc_status pxc_sync_status(pxc_workspace* ws, cudaStream_t s) {
  if (!ws) return fail(PXC_ERR_ARG, "null workspace");
  WsExtra* x = X(ws);
  cudaMemcpyAsync(x->h_err, ws->err, 4, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(PXC_ERR_CUDA, "sync: %s", cudaGetErrorString(e));
  unsigned bits = *x->h_err;
  if (bits) {
    cudaMemsetAsync(ws->err, 0, 4, s);
    cudaStreamSynchronize(s);
    const int order[] = {PXC_ERR_ID_RANGE, PXC_ERR_NONFINITE, PXC_ERR_OVERFLOW, PXC_ERR_TIMEOUT};
    const char* names[] = {"state id out of range", "non-finite input", "Boltzmann exponent overflow",
                           "bounded device wait ran out"};
    for (int i = 0; i < 4; ++i)
      if (bits & (1u << order[i])) return fail((pxc_status)order[i], "device: %s", names[i]);
  }
  return PXC_OK;
}

pxc_status pxc_partition_function(pxc_workspace* ws, const pxc_states* st, const pxc_condition* c, int32_t n_c,
                                  double* Q_out, double* dQ_out, cudaStream_t s) {
  if (!ws || !c || n_c < 1 || !Q_out) return fail(PXC_ERR_ARG, "partition_function: bad arguments");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  pxc_status r = check_states(st);
  if (r) return r;
  WsExtra* x = X(ws);
  if (n_c > x->L.max_cond) return fail(PXC_ERR_CAPACITY, "partition_function: n_c above capacity");
  std::vector<SlotP> sp(n_c);
  for (int i = 0; i < n_c; ++i) {
    if ((r = check_cond(c[i], false, st))) return r;
    sp[i] = make_slot(c[i]);
  }
  SlotP* dslot = at<SlotP>(ws, x->L.slots);
  if ((r = upload(ws, dslot, sp.data(), sizeof(SlotP) * n_c, s))) return r;
  double* qres = at<double>(ws, x->L.qres);
  launch_boltzmann(st, dslot, n_c, nullptr, 0, nullptr, at<double>(ws, x->L.qpart), qres, ws->err, s);
  for (int i = 0; i < n_c; ++i) {
    cudaMemcpyAsync(Q_out + i, qres + 4 * i, 8, cudaMemcpyDeviceToDevice, s);
    if (dQ_out) cudaMemcpyAsync(dQ_out + 2 * i, qres + 4 * i + 1, 16, cudaMemcpyDeviceToDevice, s);
  }
  ws->cache_valid = 0;
  return cuda_check("partition_function");
}

pxc_status pxc_cooling_function(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                const pxc_condition* c, int32_t n_c, double* W_out, double* Q_out, cudaStream_t s) {
  if (!ws || !c || n_c < 1 || !W_out) return fail(PXC_ERR_ARG, "cooling_function: bad arguments");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  pxc_status r;
  if ((r = check_states(st)) || (r = check_trans(tr))) return r;
  WsExtra* x = X(ws);
  if (n_c > x->L.max_cond) return fail(PXC_ERR_CAPACITY, "cooling_function: n_c above capacity");
  if (tr->n > ws->cap.max_lines || st->n > ws->cap.max_states)
    return fail(PXC_ERR_CAPACITY, "cooling_function: above workspace capacity");
  std::vector<SlotP> sp(n_c);
  for (int i = 0; i < n_c; ++i) {
    if ((r = check_cond(c[i], false, st))) return r;
    sp[i] = make_slot(c[i]);
  }
  SlotP* dslot = at<SlotP>(ws, x->L.slots);
  if ((r = upload(ws, dslot, sp.data(), sizeof(SlotP) * n_c, s))) return r;
  // the per-state rates S reuse the Boltzmann-table region (8 of its 16 bytes per state)
  double* S = at<double>(ws, x->L.srec);
  ws->cache_valid = 0;
  launch_cool_rates(tr, st, S, ws->err, s);
  double* qres = at<double>(ws, x->L.qres);
  launch_boltzmann(st, dslot, n_c, nullptr, 0, nullptr, at<double>(ws, x->L.qpart), qres, ws->err, s, S, W_out);
  if (Q_out)
    for (int i = 0; i < n_c; ++i) cudaMemcpyAsync(Q_out + i, qres + 4 * i, 8, cudaMemcpyDeviceToDevice, s);
  x->last_nseg = 0;
  return cuda_check("cooling_function");
}

pxc_status pxc_line_intensities(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                const pxc_condition* c, const pxc_grid* grid, double cutoff, double threshold,
                                double* nu_out, float* I_scaled_out, int32_t* I_exp_out, int64_t* n_kept_out,
                                cudaStream_t s) {
  if (!ws || !c || !I_exp_out) return fail(PXC_ERR_ARG, "line_intensities: bad arguments");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  pxc_status r;
  if ((r = check_states(st)) || (r = check_trans(tr)) || (r = check_cond(*c, false, st))) return r;
  if (grid && (r = check_grid(grid, cutoff))) return r;
  if (!(threshold >= 0.0)) return fail(PXC_ERR_ARG, "threshold must be >= 0");
  WsExtra* x = X(ws);
  const Layout& L = x->L;
  if (tr->n > ws->cap.max_lines || st->n > ws->cap.max_states)
    return fail(PXC_ERR_CAPACITY, "line_intensities: above workspace capacity");
  GridP gp = grid ? make_gridp(*grid, cutoff) : GridP{};
  unsigned long long* cnt = at<unsigned long long>(ws, L.counters);
  cudaMemsetAsync(cnt, 0, CNT_N * 8, s);
  run_boltzmann(ws, st, *c, 0, s, false);
  cudaMemsetAsync(at<unsigned long long>(ws, L.maxbits), 0, 8, s);
  const int64_t nblk = (tr->n + kLinesPerBlockI - 1) / kLinesPerBlockI;
  const BoundP bp = make_bound(ws, st, *c, threshold);
  launch_lines(tr, st->g, st->n, at<double2>(ws, L.srec), at<double>(ws, L.qres), gp, bp, grid ? 1 : 0, threshold, 1,
               at<uint64_t>(ws, L.key), at<double>(ws, L.Iv), nu_out, at<uint32_t>(ws, L.bcount), nblk,
               at<unsigned long long>(ws, L.maxbits), ws->err, s);
  if (nblk) launch_scan_counts(at<uint32_t>(ws, L.bcount), nblk, cnt + CNT_KEPT, s);
  int32_t* kexp = at<int32_t>(ws, L.kexp);
  launch_exponent(at<unsigned long long>(ws, L.maxbits), kexp, nullptr, 0, nullptr, 0, s);
  cudaMemcpyAsync(I_exp_out, kexp, 4, cudaMemcpyDeviceToDevice, s);
  if (I_scaled_out) launch_stick_out(at<double>(ws, L.Iv), at<uint64_t>(ws, L.key), tr->n, kexp, I_scaled_out, s);
  if (n_kept_out) cudaMemcpyAsync(n_kept_out, cnt + CNT_KEPT, 8, cudaMemcpyDeviceToDevice, s);
  x->last_nseg = 0;
  return cuda_check("line_intensities");
}

}  // extern "C"

namespace {

template <typename T>
void put(std::vector<unsigned char>& k, const T& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
  k.insert(k.end(), p, p + sizeof(T));
}

// Arguments that determine a single-condition call's kept, sorted line list (what the adjoint reads
// back), and the workspace modes that change it.
std::vector<unsigned char> list_key(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                    const pxc_condition& c, const pxc_grid* grid, const pxc_profile_args* pa,
                                    double threshold) {
  WsExtra* x = X(ws);
  std::vector<unsigned char> k;
  k.reserve(256);
  put(k, st->E); put(k, st->g); put(k, st->E_vib); put(k, st->n); put(k, st->n_vib);
  put(k, tr->upper); put(k, tr->lower); put(k, tr->A); put(k, tr->A_is_f32); put(k, tr->n);
  put(k, c.T); put(k, c.T_vib); put(k, c.P);
  put(k, grid->nu_min); put(k, grid->dnu); put(k, grid->n); put(k, grid->wl_unit);
  put(k, pa->kind); put(k, pa->cutoff); put(k, pa->mass_da); put(k, pa->hwhm); put(k, pa->gamma_ref);
  put(k, pa->n_T); put(k, pa->T_ref);
  put(k, threshold); put(k, x->emission); put(k, ws->accumulate);
  return k;
}

// Whether a call leaves a line list the adjoint may reuse (single condition, wavenumber grid, a
// kind with an adjoint, no chunk accumulation).
bool reusable_call(pxc_workspace* ws, int32_t n_c, const pxc_grid* grid, const pxc_profile_args* pa) {
  return X(ws)->reuse_fwd && n_c == 1 && grid->wl_unit == 0.0 && pa->kind <= PXC_VOIGT && !ws->accumulate &&
         !X(ws)->emission;
}

// Profile-kernel arguments over the sorted list of the call (all temperature slots' intensities).
ProfP profile_params(pxc_workspace* ws, const pxc_profile_args* pa, const pxc_grid* grid, const CondDev* dcond,
                     float* sigma_out, long long wait_limit) {
  const Layout& L = X(ws)->L;
  ProfP p{};
  p.pos = at<int4>(ws, L.pos);
  p.par = at<float2>(ws, L.par);
  p.Is = at<float>(ws, L.Is);
  p.is_stride = L.is_stride;
  p.cond = dcond;
  p.items = at<Item>(ws, L.items);
  p.n_items = at<unsigned long long>(ws, L.counters) + CNT_ITEMS;
  p.queue = at<unsigned long long>(ws, L.counters) + CNT_QUEUE;
  p.sigma = sigma_out;
  p.partial = at<float>(ws, L.partial);
  p.n_grid = grid->n;
  p.nu_min = grid->nu_min;
  p.dnu = grid->dnu;
  p.accumulate = ws->accumulate;
  p.kind = pa->kind;
  p.err = ws->err;
  p.spin_limit = wait_limit;
  p.drain_limit = kDefaultWaitLimit;  // copies in flight always land; this bound is never the one reached
  p.wl_unit = grid->wl_unit;
  return p;
}

pxc_status cross_section_direct(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                const pxc_condition* c, int32_t n_c, const pxc_grid* grid,
                                const pxc_profile_args* pa, double threshold, float* sigma_out,
                                int32_t* sigma_exp_out, cudaStream_t s) {
  if (!ws || !c || n_c < 1 || !sigma_out || !sigma_exp_out) return fail(PXC_ERR_ARG, "cross_section: bad arguments");
  pxc_status r;
  if ((r = check_states(st)) || (r = check_trans(tr)) || (r = check_prof(pa, tr))) return r;
  if ((r = check_grid(grid, pa->cutoff))) return r;
  if (!(threshold >= 0.0)) return fail(PXC_ERR_ARG, "threshold must be >= 0");
  for (int i = 0; i < n_c; ++i) {
    if ((r = check_cond(c[i], false, st))) return r;
    if (width_kind(pa->kind) == PXC_LORENTZ && !(c[i].P > 0.0)) return fail(PXC_ERR_ARG, "Lorentzian profile needs P > 0");
    if (!(c[i].P >= 0.0)) return fail(PXC_ERR_ARG, "condition: P must be >= 0");
  }
  WsExtra* x = X(ws);
  const Layout& L = x->L;
  if (tr->n > ws->cap.max_lines || st->n > ws->cap.max_states || grid->n > std::max<int64_t>(ws->cap.max_grid, 1) ||
      n_c > L.max_cond)
    return fail(PXC_ERR_CAPACITY, "cross_section: above workspace capacity");
  if (ws->accumulate && n_c != 1) return fail(PXC_ERR_ARG, "accumulate mode needs n_c == 1");
  const bool wl = grid->wl_unit > 0.0;
  if (wl && is_binned(pa->kind)) return fail(PXC_ERR_ARG, "wavelength grids take the sampled profiles only");
  const double wpts = 2.0 * pa->cutoff / grid->dnu + 2.0;
  // wavelength grids: 128-point segments (tile 0), one work item per segment
  const int tile = wl ? 0 : x->tile[pa->kind][n_c > 1 ? 1 : 0];
  const int seg = tile_seg(tile);
  const int64_t nseg = (grid->n + seg - 1) / seg;
  const int64_t max_partial = L.partial_floats / seg;
  if (!wl && n_c == 1 && wpts > kWinCap) {
    // the split-item table is sized for windows up to kWinCap points
    const int64_t need = nseg + (int64_t)((double)tr->n * (wpts / seg + 2.0) / kItemLines) + 1;
    if (need > L.max_items || need - nseg > max_partial)
      return fail(PXC_ERR_CAPACITY, "cross_section: cut-off window too wide for this workspace");
  }
  GridP gp = make_gridp(*grid, pa->cutoff);
  unsigned long long* cnt = at<unsigned long long>(ws, L.counters);
  cudaMemsetAsync(cnt, 0, CNT_N * 8, s);

  // distinct temperature slots
  std::vector<int> slot_of(n_c);
  std::vector<pxc_condition> slots;
  for (int i = 0; i < n_c; ++i) {
    int f = -1;
    for (size_t k = 0; k < slots.size(); ++k)
      if (slots[k].T == c[i].T && slots[k].T_vib == c[i].T_vib) { f = (int)k; break; }
    if (f < 0) { f = (int)slots.size(); slots.push_back(c[i]); }
    slot_of[i] = f;
  }
  if ((int64_t)slots.size() > L.max_slots) return fail(PXC_ERR_CAPACITY, "more distinct temperatures than capacity");
  std::vector<CondDev> cds(n_c);
  for (int i = 0; i < n_c; ++i) cds[i] = make_cond(c[i], *pa, slot_of[i]);
  CondDev* dcond = at<CondDev>(ws, L.cond);
  if ((r = upload(ws, dcond, cds.data(), sizeof(CondDev) * n_c, s))) return r;

  uint64_t* keys[2] = {at<uint64_t>(ws, L.skey0), at<uint64_t>(ws, L.skey1)};
  uint32_t* idxs[2] = {at<uint32_t>(ws, L.sidx0), at<uint32_t>(ws, L.sidx1)};
  int32_t* kexp = at<int32_t>(ws, L.kexp);
  if (n_c == 1) {
    // with pxc_set_reuse_forward, the sorted ids and A are gathered too, for a later adjoint
    const bool gather = reusable_call(ws, n_c, grid, pa);
    if ((r = front_plain(ws, st, tr, c[0], gp, pa, threshold, sigma_exp_out, sigma_out, grid->n, gather, s))) return r;
  } else {
    // geometry only: kept set from nu and the window; intensities per temperature slot in sorted order.
    // The geometry pass reads E through the state table, so fill it (first slot) first.
    run_boltzmann(ws, st, slots[0], 0, s, false);
    const int64_t nunit = (tr->n + kUnitLines - 1) / kUnitLines;
    BoundP bp = make_bound(ws, st, c[0], 0.0);
    launch_lines_compact(tr, st->n, at<code_t>(ws, L.code), qhdr(ws), at<StateFast>(ws, L.sfast),
                         at<double>(ws, L.qres), gp, 0.0, bp, 0, CAND_BUFFERS(ws, L),
                         at<uint64_t>(ws, L.key), idxs[1], nullptr, at<uint32_t>(ws, L.bcount), nunit, nullptr,
                         ws->err, s);
    if (nunit) launch_scan_counts(at<uint32_t>(ws, L.bcount), nunit, cnt + CNT_KEPT, s);
    launch_compact_staged(at<uint64_t>(ws, L.key), idxs[1], at<uint32_t>(ws, L.bcount), nunit, keys[0], idxs[0], s);
    launch_radix_sort(keys, idxs, cnt + CNT_KEPT, tr->n, at<uint32_t>(ws, L.rcount), s);
    launch_prepare(keys[0], idxs[0], cnt + CNT_KEPT, tr->n, gp, pa->gamma_ref, pa->n_T, nullptr, kexp,
                   at<int4>(ws, L.pos), at<float2>(ws, L.par), nullptr, tr, at<int32_t>(ws, L.su),
                   at<int32_t>(ws, L.sl), at<double>(ws, L.sA), nullptr, cnt, s);
    // conditions grouped by temperature slot (wavenumber grids: one profile launch per slot over
    // that slot's lines with non-zero scaled intensity)
    std::vector<int32_t> order;
    std::vector<int> first(slots.size() + 1, 0);
    for (size_t k = 0; k < slots.size(); ++k) {
      first[k] = (int)order.size();
      for (int i = 0; i < n_c; ++i)
        if (slot_of[i] == (int)k) order.push_back(i);
    }
    first[slots.size()] = (int)order.size();
    int32_t* condlist = at<int32_t>(ws, L.condlist);
    if (!wl && (r = upload(ws, condlist, order.data(), sizeof(int32_t) * order.size(), s))) return r;
    const int ctas_b = profile_ctas(ws, pa->kind, tile);
    for (size_t k = 0; k < slots.size(); ++k) {
      if (k) run_boltzmann(ws, st, slots[k], (int)k, s, false);
      cudaMemsetAsync(at<unsigned long long>(ws, L.maxbits) + k, 0, 8, s);
      launch_sorted_intensity(at<int32_t>(ws, L.su), at<int32_t>(ws, L.sl), at<double>(ws, L.sA), cnt + CNT_KEPT,
                              tr->n, st->g, at<double2>(ws, L.srec), at<double>(ws, L.qres) + 4 * k,
                              make_bound(ws, st, slots[k], threshold), threshold, at<double>(ws, L.sI),
                              at<unsigned long long>(ws, L.maxbits) + k, s);
      launch_exponent(at<unsigned long long>(ws, L.maxbits) + k, kexp + 2 * k, nullptr, 0, nullptr, 0, s);
      float* Is_k = at<float>(ws, L.Is) + (int64_t)k * L.is_stride;
      launch_scale(at<double>(ws, L.sI), cnt + CNT_KEPT, tr->n, kexp + 2 * k, Is_k, cnt, s);
      if (wl) continue;
      launch_compact_nonzero(at<int4>(ws, L.pos), at<float2>(ws, L.par), Is_k, cnt + CNT_KEPT, tr->n,
                             at<uint32_t>(ws, L.bcount), cnt + CNT_SLOT_NZ, at<int4>(ws, L.pos_c),
                             at<float2>(ws, L.par_c), at<float>(ws, L.Is_c), s);
      launch_segments(at<int4>(ws, L.pos_c), cnt + CNT_SLOT_NZ, nseg, seg, at<int32_t>(ws, L.segr), s);
      // segments with many lines (lines piled up at one wavenumber) are split into items of
      // similar size whose partial rows are added afterwards, as in single-condition calls
      const int mk = first[k + 1] - first[k];
      launch_items(at<int32_t>(ws, L.segr), nseg, mk, kItemLines, at<int32_t>(ws, L.seg_items),
                   at<Item>(ws, L.items), cnt, L.max_items, 16ll * ctas_b, max_partial, condlist + first[k], s);
      ProfP p = profile_params(ws, pa, grid, dcond, sigma_out, x->wait_limit);
      p.pos = at<int4>(ws, L.pos_c);
      p.par = at<float2>(ws, L.par_c);
      p.Is = at<float>(ws, L.Is_c);
      p.is_stride = 0;
      tmark(ws, 2, true, s);
      launch_profile(p, tile, ctas_b, s);
      tmark(ws, 2, false, s);
      launch_reduce_partials(at<Item>(ws, L.items), at<int32_t>(ws, L.seg_items), nseg, seg, mk,
                             at<float>(ws, L.partial), sigma_out, grid->n, condlist + first[k], s);
    }
    for (int i = 0; i < n_c; ++i)
      cudaMemcpyAsync(sigma_exp_out + i, kexp + 2 * slot_of[i], 4, cudaMemcpyDeviceToDevice, s);
    if (!wl) {
      x->last_nseg = nseg;
      x->last_seg = seg;
      x->last_tile = tile;
      ws->last_nc = n_c;
      return cuda_check("cross_section");
    }
  }
  const int ctas = profile_ctas(ws, pa->kind, tile);
  const bool split = n_c == 1 && !wl;  // only single-condition wavenumber calls split segments
  launch_segments(at<int4>(ws, L.pos), cnt + CNT_KEPT, nseg, seg, at<int32_t>(ws, L.segr), s);
  launch_items(at<int32_t>(ws, L.segr), nseg, n_c, split ? kItemLines : INT32_MAX / 2, at<int32_t>(ws, L.seg_items),
               at<Item>(ws, L.items), cnt, L.max_items, split ? 16ll * ctas : 0ll, max_partial, nullptr, s);
  ProfP p = profile_params(ws, pa, grid, dcond, sigma_out, x->wait_limit);
  tmark(ws, 2, true, s);
  if (wl) launch_profile_wl(p, (int64_t)n_c * nseg, s);
  else launch_profile(p, tile, ctas, s);
  tmark(ws, 2, false, s);
  if (n_c == 1)
    launch_reduce_partials(at<Item>(ws, L.items), at<int32_t>(ws, L.seg_items), nseg, seg, 1,
                           at<float>(ws, L.partial), sigma_out, grid->n, nullptr, s);
  x->last_nseg = nseg;
  x->last_seg = seg;
  x->last_tile = tile;
  ws->last_nc = n_c;
  return cuda_check("cross_section");
}


// Everything a captured call depends on besides the contents of device memory: the pointers and
// sizes of every array, the conditions, grid, profile and threshold, and the workspace's modes.
std::vector<unsigned char> graph_key(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                     const pxc_condition* c, int32_t n_c, const pxc_grid* grid,
                                     const pxc_profile_args* pa, double threshold, float* sigma_out,
                                     int32_t* sigma_exp_out, cudaStream_t s) {
  WsExtra* x = X(ws);
  std::vector<unsigned char> k;
  k.reserve(256 + 24 * (size_t)n_c);
  put(k, st->E); put(k, st->g); put(k, st->E_vib); put(k, st->n); put(k, st->n_vib);
  put(k, tr->upper); put(k, tr->lower); put(k, tr->A); put(k, tr->A_is_f32); put(k, tr->n);
  put(k, n_c);
  for (int i = 0; i < n_c; ++i) { put(k, c[i].T); put(k, c[i].T_vib); put(k, c[i].P); }
  put(k, grid->nu_min); put(k, grid->dnu); put(k, grid->n); put(k, grid->wl_unit);
  put(k, pa->kind); put(k, pa->cutoff); put(k, pa->mass_da); put(k, pa->hwhm); put(k, pa->gamma_ref);
  put(k, pa->n_T); put(k, pa->T_ref);
  put(k, threshold); put(k, sigma_out); put(k, sigma_exp_out);
  const int kind = pa->kind >= 0 && pa->kind < kNumKinds ? pa->kind : 0;
  put(k, x->tile[kind][n_c > 1 ? 1 : 0]); put(k, x->emission); put(k, x->wait_limit); put(k, x->reuse_fwd);
  (void)s;
  return k;
}

pxc_status launch_entry(pxc_workspace* ws, GraphEntry& g, cudaStream_t s) {
  WsExtra* x = X(ws);
  if (cudaGraphLaunch(g.exec, s) != cudaSuccess) return cuda_check("cross_section graph launch");
  note_launches((int)g.kernels);
  x->last_nseg = g.last_nseg;
  x->last_seg = g.last_seg;
  x->last_tile = g.last_tile;
  ws->last_nc = g.last_nc;
  return cuda_check("cross_section graph launch");
}

}  // namespace

extern "C" {

pxc_status pxc_set_graphs(pxc_workspace* ws, int on) {
  if (!ws) return fail(PXC_ERR_ARG, "set_graphs: null workspace");
  WsExtra* x = X(ws);
  x->graphs = on ? 1 : 0;
  if (!on) {
    for (auto& g : x->gcache) cudaGraphExecDestroy(g.exec);
    x->gcache.clear();
  }
  return cuda_check("set_graphs");
}

pxc_status pxc_graph_stats(pxc_workspace* ws, int64_t* captures, int64_t* replays, int32_t* cached) {
  if (!ws) return fail(PXC_ERR_ARG, "graph_stats: null workspace");
  WsExtra* x = X(ws);
  if (captures) *captures = x->graph_captures;
  if (replays) *replays = x->graph_hits;
  if (cached) *cached = (int32_t)x->gcache.size();
  return PXC_OK;
}

static pxc_status cross_section_graphs(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                       const pxc_condition* c, int32_t n_c, const pxc_grid* grid,
                                       const pxc_profile_args* pa, double threshold, float* sigma_out,
                                       int32_t* sigma_exp_out, cudaStream_t s) {
  WsExtra* x = X(ws);
  if (!x->graphs || ws->accumulate || x->capturing)
    return cross_section_direct(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out, s);
  std::vector<unsigned char> key = graph_key(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out, s);
  for (size_t i = 0; i < x->gcache.size(); ++i) {
    if (x->gcache[i].key == key) {
      GraphEntry g = x->gcache[i];
      x->gcache.erase(x->gcache.begin() + (long)i);
      x->gcache.push_back(g);
      ++x->graph_hits;
      return launch_entry(ws, x->gcache.back(), s);
    }
  }
  // capture the call on the workspace's own stream (the caller's may be the legacy default
  // stream, which cannot be captured), then launch the instantiated graph on the caller's
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return cuda_check("cross_section: begin capture");
  x->capturing = 1;
  const int64_t before = launches_total();
  pxc_status r = cross_section_direct(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out,
                                      x->cap_stream);
  const int64_t noted = launches_total() - before;
  note_launches((int)-noted);  // nothing ran yet: the graph's kernels are counted when it launches
  x->capturing = 0;
  const cudaError_t ee = cudaStreamEndCapture(x->cap_stream, &graph);
  if (r) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return r;
  }
  if (ee != cudaSuccess || !graph) return fail(PXC_ERR_CUDA, "cross_section: capture failed: %s", cudaGetErrorString(ee));
  GraphEntry g{};
  g.key = std::move(key);
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
  for (auto& n : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++g.kernels;
  }
  const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(PXC_ERR_CUDA, "cross_section: instantiate: %s", cudaGetErrorString(ie));
  g.last_nseg = x->last_nseg;
  g.last_seg = x->last_seg;
  g.last_tile = x->last_tile;
  g.last_nc = ws->last_nc;
  if (x->gcache.size() >= kGraphCacheMax) {
    cudaGraphExecDestroy(x->gcache.front().exec);
    x->gcache.erase(x->gcache.begin());
  }
  x->gcache.push_back(std::move(g));
  ++x->graph_captures;
  return launch_entry(ws, x->gcache.back(), s);
}

pxc_status pxc_cross_section(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                             const pxc_condition* c, int32_t n_c, const pxc_grid* grid, const pxc_profile_args* pa,
                             double threshold, float* sigma_out, int32_t* sigma_exp_out, cudaStream_t s) {
  if (!ws || !c || n_c < 1 || !sigma_out || !sigma_exp_out || !st || !tr || !grid || !pa)
    return fail(PXC_ERR_ARG, "cross_section: bad arguments");
  WsExtra* x = X(ws);
  x->fwd_key.clear();
  const pxc_status r = cross_section_graphs(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out, s);
  if (r == PXC_OK && reusable_call(ws, n_c, grid, pa)) x->fwd_key = list_key(ws, st, tr, c[0], grid, pa, threshold);
  return r;
}

pxc_status pxc_set_reuse_forward(pxc_workspace* ws, int32_t on) {
  if (!ws) return fail(PXC_ERR_ARG, "set_reuse_forward: null workspace");
  X(ws)->reuse_fwd = on ? 1 : 0;
  X(ws)->fwd_key.clear();
  return PXC_OK;
}

pxc_status pxc_cross_section_backward(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr,
                                      const pxc_condition* c, int32_t n_c, const pxc_grid* grid,
                                      const pxc_profile_args* pa, double threshold, const float* dL_dsigma,
                                      double* dL_dT, double* dL_dTvib, double* dL_dP, float* dL_dgamma_ref,
                                      float* dL_dA, cudaStream_t s) {
  if (!ws || !c || n_c != 1 || !dL_dsigma || !dL_dT) return fail(PXC_ERR_ARG, "backward: bad arguments (n_c must be 1)");
  pxc_status r;
  if ((r = check_states(st)) || (r = check_trans(tr)) || (r = check_prof(pa, tr)) || (r = check_cond(*c, false, st)))
    return r;
  if ((r = check_grid(grid, pa->cutoff))) return r;
  WsExtra* x = X(ws);
  const Layout& L = x->L;
  if (tr->n > ws->cap.max_lines || st->n > ws->cap.max_states || grid->n > std::max<int64_t>(ws->cap.max_grid, 1))
    return fail(PXC_ERR_CAPACITY, "backward: above workspace capacity");
  if (ws->accumulate) return fail(PXC_ERR_ARG, "backward: accumulate mode is forward-only");
  if (x->emission || st->n_vib)
    return fail(PXC_ERR_ARG, "backward: absorption with LTE or two-temperature populations only");
  if (pa->kind > PXC_VOIGT)
    return fail(PXC_ERR_ARG, "backward: Gaussian, Lorentzian and Voigt only (binned and pseudo-Voigt kinds are forward-only)");
  if (grid->wl_unit != 0.0) return fail(PXC_ERR_ARG, "backward: wavenumber grids only");
  GridP gp = make_gridp(*grid, pa->cutoff);
  unsigned long long* cnt = at<unsigned long long>(ws, L.counters);
  // the line list of the preceding call, when pxc_set_reuse_forward is on and its arguments match
  std::vector<unsigned char> key = list_key(ws, st, tr, *c, grid, pa, threshold);
  const bool reuse = x->reuse_fwd && !x->fwd_key.empty() && x->fwd_key == key;
  if (!reuse) {
    x->fwd_key.clear();
    cudaMemsetAsync(cnt, 0, CNT_N * 8, s);
    if ((r = front_plain(ws, st, tr, *c, gp, pa, threshold, nullptr, nullptr, grid->n, true, s))) return r;
    if (x->reuse_fwd) x->fwd_key = std::move(key);
  }
  if (dL_dA) cudaMemsetAsync(dL_dA, 0, sizeof(float) * tr->n, s);
  if (dL_dgamma_ref) cudaMemsetAsync(dL_dgamma_ref, 0, sizeof(float) * tr->n, s);
  AdjP p{};
  p.pos = at<int4>(ws, L.pos);
  p.par = at<float2>(ws, L.par);
  p.Is = at<float>(ws, L.Is);
  p.sidx = at<uint32_t>(ws, L.sidx0);
  p.su = at<int32_t>(ws, L.su);
  p.sl = at<int32_t>(ws, L.sl);
  p.sA = at<double>(ws, L.sA);
  p.srec = at<double2>(ws, L.srec);
  p.E_vib = st->E_vib;
  p.n_T = pa->n_T;
  p.qres = at<double>(ws, L.qres);
  p.w = dL_dsigma;
  p.n_dev = cnt + CNT_KEPT;
  p.n_max = tr->n;
  p.n_grid = grid->n;
  p.nu_min = grid->nu_min;
  p.dnu = grid->dnu;
  p.T = c->T;
  p.T_vib = c->T_vib > 0 ? c->T_vib : 0.0;
  p.P = c->P;
  p.T_ref = pa->T_ref;
  p.c2 = kH * kC / kKB;
  p.cond = make_cond(*c, *pa, 0);
  p.kind = pa->kind;
  p.dA = dL_dA;
  p.dgref = dL_dgamma_ref;
  // per-line scalar shares reuse buffers that are free after the sort
  p.lineT = at<double>(ws, L.key);
  p.lineTv = at<double>(ws, L.Iv);
  p.lineP = at<double>(ws, L.sI);
  launch_adjoint(p, s);
  // the Q partial sums are final by now: their buffer holds the reduction's per-CTA totals
  if (adjoint_reduce_scratch_bytes() > (size_t)kQBlocks * kQMoments * 8)
    return fail(PXC_ERR_CAPACITY, "backward: reduction scratch larger than the Q partial buffer");
  launch_adjoint_reduce(p.lineT, p.lineTv, p.lineP, cnt + CNT_KEPT, at<double>(ws, L.qpart), dL_dT, dL_dTvib, dL_dP, s);
  x->last_nseg = 0;  // the adjoint does not bin lines into segments
  ws->last_nc = 1;
  return cuda_check("cross_section_backward");
}

pxc_status pxc_get_stats(pxc_workspace* ws, cudaStream_t s, pxc_stats* out) {
  if (!ws || !out) return fail(PXC_ERR_ARG, "get_stats: bad arguments");
  WsExtra* x = X(ws);
  cudaMemcpyAsync(x->h_cnt, ws->counters, CNT_N * 8, cudaMemcpyDeviceToHost, s);
  int32_t k = 0;
  cudaMemcpyAsync(x->h_params, at<int32_t>(ws, x->L.kexp), 4, cudaMemcpyDeviceToHost, s);
  pxc_status r = pxc_sync_status(ws, s);
  memcpy(&k, x->h_params, 4);
  out->n_kept = (int64_t)x->h_cnt[CNT_KEPT];
  out->n_nonzero = (int64_t)x->h_cnt[CNT_NONZERO];
  out->evals_window = (int64_t)x->h_cnt[CNT_EVALS];
  out->evals_nonzero = (int64_t)x->h_cnt[CNT_EVALS_NZ];
  out->segment_points = x->last_seg;
  out->n_segments = (int32_t)x->last_nseg;
  out->I_exp = k;
  out->tile = x->last_tile;
  return r;
}

pxc_status pxc_set_tile(pxc_workspace* ws, int32_t kind, int32_t batched, int32_t tile) {
  if (!ws || kind < 0 || kind >= kNumKinds || batched < 0 || batched > 1 || tile < 0 || tile >= kNumTiles)
    return fail(PXC_ERR_ARG, "set_tile: bad arguments");
  X(ws)->tile[kind][batched] = tile;
  return PXC_OK;
}

pxc_status pxc_get_tile(pxc_workspace* ws, int32_t kind, int32_t batched, int32_t* tile) {
  if (!ws || !tile || kind < 0 || kind >= kNumKinds || batched < 0 || batched > 1)
    return fail(PXC_ERR_ARG, "get_tile: bad arguments");
  *tile = X(ws)->tile[kind][batched];
  return PXC_OK;
}

pxc_status pxc_autotune(pxc_workspace* ws, const pxc_states* st, const pxc_transitions* tr, const pxc_condition* c,
                        int32_t n_c, const pxc_grid* grid, const pxc_profile_args* pa, double threshold,
                        float* sigma_out, int32_t* sigma_exp_out, int32_t repeats, int32_t* tile_out,
                        double* ms_out, cudaStream_t s) {
  if (!ws || !pa || pa->kind < 0 || pa->kind >= kNumKinds || n_c < 1 || repeats < 1)
    return fail(PXC_ERR_ARG, "autotune: bad arguments");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  if (ws->accumulate) return fail(PXC_ERR_ARG, "autotune: not in accumulate mode (runs the call repeatedly)");
  WsExtra* x = X(ws);
  const int b = n_c > 1 ? 1 : 0;
  const int saved = x->tile[pa->kind][b];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_ms = 0.0;
  int best = -1;
  pxc_status r = PXC_OK;
  for (int t = 0; t < kNumTiles && !r; ++t) {
    x->tile[pa->kind][b] = t;
    r = pxc_cross_section(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out, s);
    if (r) break;
    cudaEventRecord(e0, s);
    for (int i = 0; i < repeats && !r; ++i)
      r = pxc_cross_section(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out, s);
    cudaEventRecord(e1, s);
    if (r) break;
    if ((r = pxc_sync_status(ws, s))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / repeats;
    if (ms_out) ms_out[t] = per;
    if (best < 0 || per < best_ms) { best_ms = per; best = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r || best < 0) {
    x->tile[pa->kind][b] = saved;
    return r ? r : fail(PXC_ERR_ARG, "autotune: nothing timed");
  }
  x->tile[pa->kind][b] = best;
  if (tile_out) *tile_out = best;
  // leave the chosen tile's result in the outputs
  if (best != kNumTiles - 1) r = pxc_cross_section(ws, st, tr, c, n_c, grid, pa, threshold, sigma_out, sigma_exp_out, s);
  if (!r) r = pxc_sync_status(ws, s);
  return r;
}

pxc_status pxc_get_binning(pxc_workspace* ws, int64_t* perm_out, int64_t* seg_first, int64_t* seg_last,
                           cudaStream_t s) {
  if (!ws) return fail(PXC_ERR_ARG, "get_binning: null workspace");
  WsExtra* x = X(ws);
  const Layout& L = x->L;
  cudaMemcpyAsync(x->h_cnt, ws->counters, CNT_N * 8, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(PXC_ERR_CUDA, "get_binning: %s", cudaGetErrorString(e));
  const int64_t n = (int64_t)x->h_cnt[CNT_KEPT];
  const int64_t nseg = x->last_nseg;
  std::vector<uint32_t> idx(n);
  std::vector<int32_t> seg(2 * nseg);
  if (n) cudaMemcpy(idx.data(), at<uint32_t>(ws, L.sidx0), 4 * n, cudaMemcpyDeviceToHost);
  if (nseg) cudaMemcpy(seg.data(), at<int32_t>(ws, L.segr), 8 * nseg, cudaMemcpyDeviceToHost);
  std::vector<int64_t> tmp(std::max<int64_t>(n, 2 * nseg));
  if (perm_out && n) {
    for (int64_t j = 0; j < n; ++j) tmp[j] = idx[j];
    cudaMemcpy(perm_out, tmp.data(), 8 * n, cudaMemcpyHostToDevice);
  }
  if (seg_first && nseg) {
    for (int64_t j = 0; j < nseg; ++j) tmp[j] = seg[j];
    cudaMemcpy(seg_first, tmp.data(), 8 * nseg, cudaMemcpyHostToDevice);
  }
  if (seg_last && nseg) {
    for (int64_t j = 0; j < nseg; ++j) tmp[j] = seg[nseg + j];
    cudaMemcpy(seg_last, tmp.data(), 8 * nseg, cudaMemcpyHostToDevice);
  }
  return cuda_check("get_binning");
}

pxc_status pxc_set_timing(pxc_workspace* ws, int on) {
  if (!ws) return fail(PXC_ERR_ARG, "set_timing: null workspace");
  WsExtra* x = X(ws);
  if (on && x->ev_pool.empty()) {
    x->ev_pool.resize(4096);
    for (auto& e : x->ev_pool) cudaEventCreate(&e);
  }
  x->timing = on ? 1 : 0;
  x->ev_used.clear();
  x->ev_next = 0;
  return cuda_check("set_timing");
}

pxc_status pxc_get_timing(pxc_workspace* ws, cudaStream_t s, double* ms, int64_t* count) {
  if (!ws || !ms) return fail(PXC_ERR_ARG, "get_timing: bad arguments");
  WsExtra* x = X(ws);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(PXC_ERR_CUDA, "get_timing: %s", cudaGetErrorString(e));
  for (int i = 0; i < 3; ++i) { ms[i] = 0.0; if (count) count[i] = 0; }
  for (auto& u : x->ev_used) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, x->ev_pool[u.second], x->ev_pool[u.second + 1]) == cudaSuccess) {
      ms[u.first] += t;
      if (count) count[u.first] += 1;
    }
  }
  x->ev_used.clear();
  x->ev_next = 0;
  return cuda_check("get_timing");
}

size_t pxc_stream_buffer_bytes(int64_t chunk_lines, int32_t A_is_f32, int32_t with_broadening) {
  size_t per = 8 + (A_is_f32 ? 4 : 8) + (with_broadening ? 8 : 0);
  return al((size_t)chunk_lines * per) + 5 * 256;
}

__global__ void k_set_int(int32_t* p, int32_t v) { *p = v; }

pxc_status pxc_cross_section_streamed(pxc_workspace* ws, const pxc_states* st, const int32_t* h_up,
                                      const int32_t* h_lo, const void* h_A, int32_t A_is_f32, const float* h_gref,
                                      const float* h_nT, int64_t n_lines, const pxc_condition* c,
                                      const pxc_grid* grid, const pxc_profile_args* pa, double threshold,
                                      void* buf0, void* buf1, size_t buf_bytes, float* sigma_out,
                                      int32_t* sigma_exp_out, cudaStream_t s) {
  if (!ws || !h_up || !h_lo || !h_A || n_lines < 0 || !c || !grid || !pa || !buf0 || !buf1 || !sigma_out ||
      !sigma_exp_out)
    return fail(PXC_ERR_ARG, "streamed: bad arguments");
  X(ws)->fwd_key.clear();  // the workspace no longer holds a reusable line list
  const int wk = width_kind(pa->kind);
  const bool broad = wk == PXC_LORENTZ || wk == PXC_VOIGT;
  if (broad && (!h_gref || !h_nT)) return fail(PXC_ERR_ARG, "streamed: gamma_ref and n_T required");
  const int64_t chunk = ws->cap.max_lines;
  if (chunk < 1) return fail(PXC_ERR_CAPACITY, "streamed: workspace has no line capacity");
  if (buf_bytes < pxc_stream_buffer_bytes(chunk, A_is_f32, broad)) return fail(PXC_ERR_CAPACITY, "streamed: buffers too small");
  WsExtra* x = X(ws);
  void* bufs[2] = {buf0, buf1};
  const size_t asz = A_is_f32 ? 4 : 8;
  int prev_acc = ws->accumulate;
  ws->accumulate = 1;
  ws->cache_valid = 0;
  cudaMemsetAsync(sigma_out, 0, sizeof(float) * grid->n, s);
  k_set_int<<<1, 1, 0, s>>>(sigma_exp_out, PXC_EXP_EMPTY);
  note_launches(1);
  pxc_status r = PXC_OK;
  const int64_t nchunks = (n_lines + chunk - 1) / chunk;
  // make the copy stream see everything issued so far on `s`
  cudaEventRecord(x->ev_done[0], s);
  cudaEventRecord(x->ev_done[1], s);
  for (int64_t ci = 0; ci < nchunks && r == PXC_OK; ++ci) {
    const int b = (int)(ci & 1);
    const int64_t t0 = ci * chunk, n = std::min(chunk, n_lines - t0);
    char* base = (char*)bufs[b];
    int32_t* d_up = (int32_t*)base;
    int32_t* d_lo = (int32_t*)(base + al(4 * chunk));
    char* d_A = base + 2 * al(4 * chunk);
    float* d_g = (float*)(d_A + al(asz * chunk));
    float* d_n = (float*)((char*)d_g + al(4 * chunk));
    cudaStreamWaitEvent(x->copy_stream, x->ev_done[b], 0);
    cudaMemcpyAsync(d_up, h_up + t0, 4 * n, cudaMemcpyHostToDevice, x->copy_stream);
    cudaMemcpyAsync(d_lo, h_lo + t0, 4 * n, cudaMemcpyHostToDevice, x->copy_stream);
    cudaMemcpyAsync(d_A, (const char*)h_A + asz * t0, asz * n, cudaMemcpyHostToDevice, x->copy_stream);
    if (broad) {
      cudaMemcpyAsync(d_g, h_gref + t0, 4 * n, cudaMemcpyHostToDevice, x->copy_stream);
      cudaMemcpyAsync(d_n, h_nT + t0, 4 * n, cudaMemcpyHostToDevice, x->copy_stream);
    }
    cudaEventRecord(x->ev_copied[b], x->copy_stream);
    cudaStreamWaitEvent(s, x->ev_copied[b], 0);
    pxc_transitions tr{d_up, d_lo, d_A, A_is_f32, n};
    pxc_profile_args pc = *pa;
    pc.gamma_ref = broad ? d_g : nullptr;
    pc.n_T = broad ? d_n : nullptr;
    r = pxc_cross_section(ws, st, &tr, c, 1, grid, &pc, threshold, sigma_out, sigma_exp_out, s);
    cudaEventRecord(x->ev_done[b], s);
  }
  ws->accumulate = prev_acc;
  ws->cache_valid = 0;
  if (r) return r;
  return cuda_check("cross_section_streamed");
}

}  // extern "C"
