// Instruction-throughput microbenchmark of the current device: FP32 FMA, MUFU reciprocal,
// MUFU exp2, and the profile kernel's far-wing evaluation mix (five FP32 FMAs and one MUFU
// reciprocal per line-grid evaluation).  The profile pass is bound by these pipes, so its
// roofline is stated against rates measured here rather than against datasheet figures.
//
// Each kernel runs one full wave (the device's resident-CTA limit on every SM) of threads that
// iterate kChains independent dependency chains, so every pipe has enough independent work in
// flight.  Thread 0 of every CTA records its SM and the SM clock at the start and end of its
// loop; each SM's rate is the work of its CTAs over the span of their cycle counts (one clock per
// SM), independent of the clock frequency.  CUDA events give the absolute rate at the clock the
// device ran.
#include <algorithm>
#include <climits>
#include <vector>

#include "kernels.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kDiagThreads = 256;

__device__ __forceinline__ float d_rcp(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float d_ex2(float x) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// mode 0: kChains FMAs per iteration; 1: kChains reciprocals (each of the previous result times
// p, so no pair of reciprocals can be folded away); 2: kChains exp2;
// 3: kChains evaluations of v = x^2 + c1, den = v^2 + e, num = K v + K, acc += num / den with
//    x advanced by one FMA (5 FMAs + 1 reciprocal each)
template <int MODE>
__global__ void __launch_bounds__(kDiagThreads) k_pipe(int iters, float p, float q, float* sink,
                                                       long long* rec) {
  float a[kChains], acc[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    a[j] = 1.0f + 1e-3f * (float)(threadIdx.x + j);
    acc[j] = 0.f;
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      if (MODE == 0) {
        a[j] = fmaf(a[j], p, q);
      } else if (MODE == 1) {
        a[j] = d_rcp(a[j] * p);
      } else if (MODE == 2) {
        a[j] = d_ex2(-a[j]);
      } else {
        a[j] = fmaf(1.0f, p, a[j]);            // x advances by one step
        const float v = fmaf(a[j], a[j], q);  // x^2 + c1
        const float den = fmaf(v, v, p);      // v^2 + e
        const float num = fmaf(v, p, p);      // K v + K
        acc[j] = fmaf(num, d_rcp(den), acc[j]);
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j] + acc[j];
  if (s == 12345.678f) sink[threadIdx.x] = s;  // keeps the chains live; never true for these inputs
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    rec[3 * blockIdx.x] = sm;
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = t1;
  }
}

template <int MODE>
void launch_pipe(int blocks, int iters, float* sink, long long* rec, cudaStream_t s) {
  // the chain constants keep every value finite: FMA converges to q / (1 - p), rcp alternates,
  // exp2(-x) stays in (0.5, 1), and the evaluation mix grows x by p per step
  const float p = MODE == 3 ? 1e-3f : 0.999f, q = MODE == 3 ? 0.25f : 1e-3f;
  k_pipe<MODE><<<blocks, kDiagThreads, 0, s>>>(iters, p, q, sink, rec);
}

}  // namespace

extern "C" size_t pxc_pipe_rates_buffer_bytes(void) {
  return 3 * 4096 * sizeof(long long) + kDiagThreads * sizeof(float);
}

extern "C" pxc_status pxc_pipe_rates(void* dev_buf, size_t bytes, double* out, cudaStream_t stream) {
  if (!dev_buf || !out || bytes < pxc_pipe_rates_buffer_bytes()) {
    pxc::set_last_error("pipe_rates: null pointer or buffer below pxc_pipe_rates_buffer_bytes()");
    return PXC_ERR_ARG;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    pxc::set_last_error("pipe_rates: no usable device");
    return PXC_ERR_CUDA;
  }
  long long* cyc = static_cast<long long*>(dev_buf);
  float* sink = reinterpret_cast<float*>(cyc + 3 * 4096);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters[4] = {1 << 14, 1 << 13, 1 << 13, 1 << 12};
  const double ops_per_iter[4] = {kChains, kChains, kChains, kChains};
  std::vector<long long> h;
  for (int m = 0; m < 4; ++m) {
    int per_sm = 0;
    if (m == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pipe<0>, kDiagThreads, 0);
    if (m == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pipe<1>, kDiagThreads, 0);
    if (m == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pipe<2>, kDiagThreads, 0);
    if (m == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pipe<3>, kDiagThreads, 0);
    if (per_sm < 1) per_sm = 1;
    int blocks = sms * per_sm;
    if (blocks > 4096) blocks = 4096;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms the clocks up
      cudaEventRecord(e0, stream);
      if (m == 0) launch_pipe<0>(blocks, iters[m], sink, cyc, stream);
      if (m == 1) launch_pipe<1>(blocks, iters[m], sink, cyc, stream);
      if (m == 2) launch_pipe<2>(blocks, iters[m], sink, cyc, stream);
      if (m == 3) launch_pipe<3>(blocks, iters[m], sink, cyc, stream);
      cudaEventRecord(e1, stream);
      pxc::note_launches(1);
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      pxc::set_last_error("pipe_rates: kernel failed");
      return PXC_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h.resize(3 * (size_t)blocks);
    cudaMemcpy(h.data(), cyc, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost);
    // per SM: its CTAs' work over the span of their cycle counters
    std::vector<long long> lo(1024, LLONG_MAX), hi(1024, LLONG_MIN);
    std::vector<int> cnt(1024, 0);
    for (int b = 0; b < blocks; ++b) {
      const long long sm = h[3 * b];
      if (sm < 0 || sm >= 1024) continue;
      lo[sm] = std::min(lo[sm], h[3 * b + 1]);
      hi[sm] = std::max(hi[sm], h[3 * b + 2]);
      ++cnt[sm];
    }
    const double per_cta = (double)kDiagThreads * iters[m] * ops_per_iter[m];
    double rate = 0.0;
    int used = 0;
    for (int sm = 0; sm < 1024; ++sm) {
      if (!cnt[sm] || hi[sm] <= lo[sm]) continue;
      rate += cnt[sm] * per_cta / (double)(hi[sm] - lo[sm]);
      ++used;
    }
    out[m] = used ? rate / used : 0.0;        // results per SM per clock cycle
    out[4 + m] = (double)blocks * per_cta / (ms * 1e-3);  // results per second at the running clock
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    pxc::set_last_error(cudaGetErrorString(e));
    return PXC_ERR_CUDA;
  }
  return PXC_OK;
}
