// Partition functions without any allocation: pxc_partition_function_noalloc.
//
// Who needs this: code that may not allocate device memory at all -- a plug-in
// living inside a host application that owns every byte of device memory, a
// real-time or latency-critical path where cudaMalloc's implicit device
// synchronisation is not acceptable, or a caller that has no place to keep a
// workspace.  pxc_partition_function needs a workspace carved from caller
// memory; this variant needs none.  Its scratch (the per-condition constants,
// the per-block partial sums, the results and an error word) lives in one
// file-scope __device__ array that every GPU loading this library holds until
// the process exits.
//
// Limits and sharing rules:
//  - at most kNoAllocConditions (64) conditions per call, else PXC_ERR_CAPACITY;
//  - every call uses the same array, so calls that overlap on the GPU (two
//    streams, or two host threads) race and must be serialised by the caller;
//  - the array keeps the previous call's contents: the error word is cleared at
//    the start of each call, and every partial sum and result is written before
//    it is read, so nothing else has to start at zero;
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before capturing a stream into a CUDA graph.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr int kNoAllocConditions = 64;
constexpr int kMaxDevices = 64;

// Scratch layout, in doubles: partials [kQBlocks][64][kQMoments], results [64][4],
// condition constants [64] SlotP (4 doubles each), error word.
constexpr size_t kPartDoubles = (size_t)pxc::kQBlocks * kNoAllocConditions * pxc::kQMoments;
constexpr size_t kResDoubles = (size_t)kNoAllocConditions * 4;
constexpr size_t kSlotDoubles = (size_t)kNoAllocConditions * sizeof(pxc::SlotP) / sizeof(double);
constexpr size_t kScratchDoubles = kPartDoubles + kResDoubles + kSlotDoubles + 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct NoAllocConds {
  pxc::SlotP s[kNoAllocConditions];
  int n;
};

// Writes the condition constants into the scratch and clears the error word.
__global__ void k_noalloc_setup(const __grid_constant__ NoAllocConds conds, pxc::SlotP* slots, unsigned* err) {
  for (int i = threadIdx.x; i < conds.n; i += blockDim.x) slots[i] = conds.s[i];
  if (threadIdx.x == 0) *err = 0u;
}

// Copies Q, dQ and the latched error bits from the scratch to the caller's outputs.
__global__ void k_noalloc_out(const double* res, int n, const unsigned* err, double* Q_out, double* dQ_out,
                              int32_t* status_out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Q_out[i] = res[4 * i];
    if (dQ_out) {
      dQ_out[2 * i] = res[4 * i + 1];
      dQ_out[2 * i + 1] = res[4 * i + 2];
    }
  }
  if (threadIdx.x == 0 && status_out) {
    const unsigned b = *err;
    *status_out = (b & (1u << PXC_ERR_NONFINITE)) ? PXC_ERR_NONFINITE
                  : (b & (1u << PXC_ERR_OVERFLOW)) ? PXC_ERR_OVERFLOW
                                                   : PXC_OK;
  }
}

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" pxc_status pxc_partition_function_noalloc(const pxc_states* states, const pxc_condition* c, int32_t n_c,
                                                     double* Q_out, double* dQ_out, int32_t* status_out,
                                                     cudaStream_t stream) {
  if (!c || !Q_out || n_c < 1) {
    pxc::set_last_error("partition_function_noalloc: bad arguments");
    return PXC_ERR_ARG;
  }
  // the same checks as pxc_partition_function: states (null pointers, n < 0, more than 2^31-1
  // states) and every condition (T finite and > 0, T_vib finite, E_vib present for T_vib > 0,
  // vibronic densities only with E_vib and without T_vib)
  pxc_status r = pxc::validate_states(states);
  if (r) return r;
  if (n_c > kNoAllocConditions) {
    pxc::set_last_error("partition_function_noalloc: more than 64 conditions");
    return PXC_ERR_CAPACITY;
  }
  NoAllocConds conds{};
  conds.n = n_c;
  for (int i = 0; i < n_c; ++i) {
    if ((r = pxc::validate_condition(c[i], states))) return r;
    conds.s[i] = pxc::slot_constants(c[i]);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    pxc::set_last_error("partition_function_noalloc: no usable current device");
    return PXC_ERR_CUDA;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        pxc::set_last_error("partition_function_noalloc: cudaGetSymbolAddress failed");
        return PXC_ERR_CUDA;
      }
      g_addr[dev] = static_cast<double*>(p);
    }
    base = g_addr[dev];
  }
  double* part = base;
  double* res = part + kPartDoubles;
  pxc::SlotP* slots = reinterpret_cast<pxc::SlotP*>(res + kResDoubles);
  unsigned* err = reinterpret_cast<unsigned*>(res + kResDoubles + kSlotDoubles);
  k_noalloc_setup<<<1, 64, 0, stream>>>(conds, slots, err);
  pxc::launch_boltzmann(states, slots, n_c, nullptr, 0, nullptr, part, res, err, stream);
  k_noalloc_out<<<1, 64, 0, stream>>>(res, n_c, err, Q_out, dQ_out, status_out);
  pxc::note_launches(2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    pxc::set_last_error(cudaGetErrorString(e));
    return PXC_ERR_CUDA;
  }
  return PXC_OK;
}
