// Allocation-free rANS decoding (pw_rans_decode_noalloc).
//
// Some callers cannot allocate device memory while they decode: a plug-in
// that runs inside a host application's fixed device-memory budget, or a
// real-time pipeline that must never stall on cudaMalloc / cudaFree (cudaFree
// synchronises the whole device). This entry point decodes rANS chunks like
// pw_rans_decode but takes only device pointers from the caller and keeps
// everything else it needs (the CDF table bank, the per-chunk descriptors and
// a status word) in one file-scope device array of fixed size, so it calls no
// allocator at all.
//
// The array is shared by every call on a device and keeps the contents of
// the last call; the status word is cleared at the start of each call. Calls
// whose work overlaps on the GPU (for example on two streams at once) race on
// the array and must be serialised by the caller.
#include <mutex>

#include "ctx_kernels.cuh"
#include "pw_internal.cuh"

namespace pw {

// Scratch layout: [0, 256) status word, [256, 256 + 512 KiB) CDF table bank,
// its 64 KiB coarse level, then kNoAllocMaxChunks decode descriptors.
constexpr int kNoAllocMaxChunks = 16384;
constexpr size_t kBankBytes = (size_t)kNTables * (kNSym + 1) * sizeof(uint16_t);
constexpr size_t kCoarseBytes = (size_t)kNTables * kCoarse * sizeof(uint16_t);
constexpr size_t kDescOff = 256 + kBankBytes + kCoarseBytes;
constexpr size_t kScratchBytes = kDescOff + (size_t)kNoAllocMaxChunks * sizeof(DecChunk);

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

// Descriptors from the caller's device arrays: exclusive prefix sum of the
// symbol counts (one block), bounds of every chunk checked against the
// payload size.
__global__ void k_noalloc_descs(const uint8_t *payload, uint64_t payload_bytes, int nchunks,
                                const uint32_t *offset, const uint32_t *nbytes,
                                const uint32_t *count, const uint32_t *lanes, DecChunk *desc,
                                uint32_t *status) {
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  const int per = (nchunks + blockDim.x - 1) / blockDim.x;
  const int c0 = t * per, c1 = min(nchunks, c0 + per);
  uint32_t s = 0;
  for (int c = c0; c < c1; ++c) s += count[c];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    uint32_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t first = part[t] - s;
  for (int c = c0; c < c1; ++c) {
    DecChunk d;
    const uint64_t end = (uint64_t)offset[c] + nbytes[c];
    const bool ok = end <= payload_bytes && lanes[c] >= 1 && lanes[c] <= 32;
    d.data = ok ? payload + offset[c] : nullptr;
    d.nbytes = ok ? nbytes[c] : 0;  // a zero-length chunk is reported as corrupt
    d.count = count[c];
    d.first = first;
    d.lanes = (uint16_t)(ok ? lanes[c] : 1);
    d.plane = 0;
    desc[c] = d;
    if (!ok) atomicOr(status, kStCorrupt);
    first += count[c];
  }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and kept for the life of the process. A cudaDeviceReset
// while the library is loaded would leave a stale address here: this entry
// point does not support one.
static std::mutex g_mu;
static uint8_t *g_addr[64] = {};

static int scratch_address(uint8_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_last_error("no current CUDA device");
    return PW_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return PW_ECUDA;
    }
    g_addr[dev] = static_cast<uint8_t *>(p);
  }
  *out = g_addr[dev];
  return PW_OK;
}

}  // namespace pw

using namespace pw;

extern "C" int pw_rans_decode_noalloc(void *cuda_stream, const uint8_t *payload,
                                      size_t payload_bytes, int nchunks,
                                      const uint32_t *offset, const uint32_t *nbytes,
                                      const uint32_t *count, const uint32_t *lanes,
                                      const uint32_t *idx, int32_t *out) {
  if (nchunks < 0 || nchunks > kNoAllocMaxChunks) {
    set_last_error("pw_rans_decode_noalloc: at most 16384 chunks per call");
    return PW_EINVAL;
  }
  if (nchunks == 0) return PW_OK;
  if (!payload || !offset || !nbytes || !count || !lanes || !idx || !out) {
    set_last_error("pw_rans_decode_noalloc: null device pointer");
    return PW_EINVAL;
  }
  uint8_t *base = nullptr;
  int s = scratch_address(&base);
  if (s) return s;
  launch_failed() = false;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  uint32_t *status = reinterpret_cast<uint32_t *>(base);
  uint16_t *bank = reinterpret_cast<uint16_t *>(base + 256);
  uint16_t *coarse = reinterpret_cast<uint16_t *>(base + 256 + kBankBytes);
  DecChunk *desc = reinterpret_cast<DecChunk *>(base + kDescOff);
  if (cudaMemsetAsync(status, 0, sizeof(uint32_t), st) != cudaSuccess) {
    set_last_error("pw_rans_decode_noalloc: cudaMemsetAsync failed");
    return PW_ECUDA;
  }
  launch_cdf_bank(bank, coarse, st);
  k_noalloc_descs<<<1, 1024, 0, st>>>(payload, payload_bytes, nchunks, offset, nbytes, count,
                                      lanes, desc, status);
  launch_rans_decode(desc, nchunks, bank, coarse, idx, 0, out, 0, 0, 0, -1, status, st);
  uint32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("CUDA: ") + cudaGetErrorString(e));
    return PW_ECUDA;
  }
  if (launch_failed()) {
    launch_failed() = false;
    return PW_EUNSUPPORTED;
  }
  // every bit the decoder can set, as the context entry points report them
  if (h & kStCorrupt) {
    set_last_error("corrupt or truncated rANS chunk (or a chunk outside the payload)");
    return PW_ECORRUPT;
  }
  if (h & kStRange) {
    set_last_error("value outside the coder's range");
    return PW_EINVAL;
  }
  if (h & kStTimeout) {
    set_last_error("the decoder's bounded wait for its table copy expired");
    return PW_ETIMEOUT;
  }
  if (h) {
    set_last_error("unexpected decoder status");
    return PW_ECUDA;
  }
  return PW_OK;
}
