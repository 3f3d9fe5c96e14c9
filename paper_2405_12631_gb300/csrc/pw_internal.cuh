// Internal declarations shared by the libpwave translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pwave.h"

// ---------------------------------------------------------------------------
// Entropy-coding constants (Section 3.1: Laplace model; the coder is rANS).
namespace pw {

constexpr int kT = 62;                 // residuals -T..T coded directly
constexpr int kNSym = 2 * kT + 3;      // + ESC_L (0) and ESC_R (126)
constexpr int kLogM = 15;
constexpr uint32_t kM = 1u << kLogM;   // total frequency
constexpr uint32_t kRansL = 1u << 16;  // lower end of the state interval
constexpr int kNPhi = 16, kNJ = 128;
constexpr int kNTables = kNPhi * kNJ;  // 2048 tables of kNSym + 1 entries
constexpr int kCoarse = 16;            // coarse CDF entries per table (every 8th)
constexpr int kMixRow = kNSym + 1 + kCoarse;  // per-symbol table row: 128 entries + coarse
constexpr int kMaxLanes = 32;
constexpr int kMaxEscBits = 30;        // Exp-Golomb prefix length limit

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their memory is visible (returns at once when the
// launch carried no programmatic dependency); let the next kernel of the
// stream be scheduled once every CTA of this grid has signalled or exited.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `k` with a programmatic dependency on the previous kernel of the
// stream: it may be scheduled while that kernel finishes, so `k` must call
// griddep_wait before it touches memory an earlier kernel writes. Errors
// surface through cudaGetLastError as for a <<<>>> launch.
template <typename... P, typename... A>
inline cudaError_t launch_dep(void (*k)(P...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Kernel attributes and device properties belong to one device, so the
// launchers' one-time set-up is kept per device ordinal (0..63; others redo
// it every time). once_per_device runs f the first time it is reached with
// the current device active; two threads racing there may both run f, which
// is why f must be idempotent (setting a kernel attribute is).
inline int current_device() {
  int d = 0;
  return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}
template <typename F>
inline void once_per_device(std::atomic<uint64_t> &done, F &&f) {
  const int d = current_device();
  const uint64_t bit = (d >= 0 && d < 64) ? (1ull << d) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  f();
  if (bit) done.fetch_or(bit, std::memory_order_release);
}
// Number of SMs of the current device (cached per device).
inline int sm_count() {
  static std::atomic<int> cache[64];
  const int d = current_device();
  if (d >= 0 && d < 64) {
    const int n = cache[d].load(std::memory_order_relaxed);
    if (n) return n;
  }
  int n = 0;
  if (d < 0 || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess ||
      n <= 0)
    n = 148;
  if (d >= 0 && d < 64) cache[d].store(n, std::memory_order_relaxed);
  return n;
}

// Device status word bits (OR-ed by kernels, read by the host).
enum : uint32_t {
  kStCorrupt = 1u,     // rANS stream inconsistent (overrun / bad final state)
  kStHeader = 2u,      // stream header does not match the decode plan
  kStRange = 4u,       // a value fell outside its representable range
  kStTimeout = 8u      // a kernel's bounded wait expired
};

// ---------------------------------------------------------------------------
// Entropy-parameter -> table index (FP32 definition, identical on all sides):
//   t = rint(16 mu) clamped to +-2^23, sigma = softplus(rho),
//   j = clamp((bits(sigma) - bits(0.125)) >> 20, 0, 127),
//   packed = ((t + 2^23) << 7) | j.
__device__ __forceinline__ uint32_t pack_index(float mu, float rho) {
  float sg = rho > 20.f ? rho : log1pf(expf(rho));
  float t = rintf(__fmul_rn(mu, 16.f));
  t = fminf(fmaxf(t, -8388608.f), 8388608.f);
  int ti = (int)t;
  int b = __float_as_int(sg);
  int j = (b - 0x3E000000) >> 20;
  j = min(max(j, 0), kNJ - 1);
  return ((uint32_t)(ti + (1 << 23)) << 7) | (uint32_t)j;
}

__host__ __device__ __forceinline__ void unpack_index(uint32_t v, int &ctr, int &tid) {
  int t = (int)(v >> 7) - (1 << 23);
  int j = (int)(v & 127u);
  ctr = (t + 8) >> 4;                 // floor((t + 8) / 16)
  int phi = t - 16 * ctr;             // -8..7
  tid = (phi + 8) * kNJ + j;
}

// ---------------------------------------------------------------------------
// Step pattern of the four-step context model (Section 3.2, "wide
// checkerboard", period 2 rows x 4 columns): column phase of step k.
__host__ __device__ __forceinline__ int step_phase(int k, int row_odd) {
  // even rows: step0 x%4==0, step1 ==2, step2 ==1, step3 ==3
  // odd rows:  step0 x%4==2, step1 ==0, step2 ==3, step3 ==1
  const int even = (0) | (2 << 2) | (1 << 4) | (3 << 6);
  const int odd = (2) | (0 << 2) | (3 << 4) | (1 << 6);
  return ((row_odd ? odd : even) >> (2 * k)) & 3;
}
__host__ __device__ __forceinline__ int step_of(int y, int x) {
  const int ev[4] = {0, 2, 1, 3};   // x % 4 -> step (even rows)
  const int od[4] = {1, 3, 0, 2};   // x % 4 -> step (odd rows)
  return (y & 1) ? od[x & 3] : ev[x & 3];
}
__host__ __device__ __forceinline__ int row_count(int w, int a) {
  return w > a ? (w - a + 3) >> 2 : 0;
}
// Number of step-k positions in an h x w subband.
__host__ __device__ __forceinline__ int step_count(int h, int w, int k) {
  int ne = row_count(w, step_phase(k, 0)), no = row_count(w, step_phase(k, 1));
  return ne * ((h + 1) >> 1) + no * (h >> 1);
}
// q-th step-k position (raster order) -> (y, x)
__host__ __device__ __forceinline__ void step_pos(int w, int k, int q, int &y, int &x) {
  int ae = step_phase(k, 0), ao = step_phase(k, 1);
  int ne = row_count(w, ae), no = row_count(w, ao);
  int pair = ne + no;
  int y2 = q / pair, r = q - y2 * pair;
  if (r < ne) { y = 2 * y2; x = ae + 4 * r; }
  else { y = 2 * y2 + 1; x = ao + 4 * (r - ne); }
}
// (y, x) of step k -> q
__host__ __device__ __forceinline__ int step_index(int w, int k, int y, int x) {
  int ae = step_phase(k, 0), ao = step_phase(k, 1);
  int ne = row_count(w, ae), no = row_count(w, ao);
  return (y >> 1) * (ne + no) + ((y & 1) ? ne + ((x - ao) >> 2) : ((x - ae) >> 2));
}

// Interleaved states of a chunk of n symbols: one per 2^shift symbols
// (shift 7 by default; the stream header records it), 1..32.
constexpr int kLaneShift = 7;
__host__ __device__ __forceinline__ int chunk_lanes(int n, int shift = kLaneShift) {
  int l = n >> shift;
  return l < 1 ? 1 : (l > kMaxLanes ? kMaxLanes : l);
}

// ---------------------------------------------------------------------------
// Host-side helpers shared by the translation units.
struct Launch {
  static uint64_t *counter;  // per-context launch counter (set by the ctx)
};

}  // namespace pw

// Error reporting helpers (host).
#define PW_CUDA_TRY(expr)                                                   \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) {                                                \
      pw::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); \
      return PW_ECUDA;                                                      \
    }                                                                       \
  } while (0)

namespace pw {
void set_last_error(const std::string &s);
}
