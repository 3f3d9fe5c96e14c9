// Integer entropy-coding kernels: the Laplace CDF table bank and the
// warp-interleaved rANS decoder / encoder.
//
// The paper codes every quantised coefficient with a Laplace distribution
// whose mean and scale come from the context model, using adaptive
// arithmetic coding (Section 3.1). Encoder and decoder must agree bit for
// bit on every frequency table, so the tables are defined by a fixed
// sequence of FP32 operations:
//   table (phi, j), phi in [-8, 7], j in [0, 127]: mean phi / 16, scale
//   b_j = float with bits 0x3E000000 + (j << 20) + (1 << 19);
//   F(u) = exp(u / b) / 2 (u < 0), 1 - exp(-u / b) / 2 (u >= 0) at the 126
//   symbol edges u = k - 62.5 - phi / 16; p = differences of F with the two
//   tails as escape symbols; f = 1 + floor(max(p, 0) * (M - 127)); the
//   signed remainder M - sum f goes to the first largest f.
// exp() here is the library's own routine (Cody-Waite reduction by ln 2 and a
// degree-6 Taylor polynomial in Horner order) written with explicitly
// rounded intrinsics, so no contraction or library-specific rounding enters.
#include <atomic>
#include <mutex>

#include "pw_internal.cuh"
#include "ctx_kernels.cuh"
#include "spec_math.cuh"
#include "cdf_warp.cuh"
#include "tc_ptx.cuh"

namespace pw {

// One warp per table. Lane l owns symbols 4l .. 4l+3 (127 symbols) and the
// CDF entries 4l .. 4l+3 (128 entries: cdf[0] = 0 .. cdf[127] = M).
// coarse (optional): every 8th CDF entry of each table, [table][16], the
// first level of the decoder's symbol search.
__global__ void k_cdf_bank(uint16_t *__restrict__ bank, uint16_t *__restrict__ coarse) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= kNTables) return;
  const int phi = warp / kNJ - 8;
  const int j = warp % kNJ;
  const float mup = __fdiv_rn((float)phi, 16.f);
  const float b = __int_as_float(0x3E000000 + (j << 20) + (1 << 19));
  const float inv_b = __fdiv_rn(1.f, b);
  // F at edges e = 0..125 (edge e separates symbol e and e+1)
  float F[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int e = 4 * lane + i;
    float u = __fsub_rn(__fsub_rn((float)e, 62.5f), mup);
    float z = __fmul_rn(u, inv_b);
    float v;
    if (u < 0.f) v = __fmul_rn(0.5f, exp32_spec(z));
    else v = __fsub_rn(1.f, __fmul_rn(0.5f, exp32_spec(-z)));
    F[i] = (e < kNSym - 1) ? v : 1.f;
  }
  int f[4];
  int run = warp_cdf(F, lane, f);
  uint16_t *row = bank + (size_t)warp * (kNSym + 1);
  if (coarse && (lane & 1) == 0) coarse[(size_t)warp * kCoarse + (lane >> 1)] = (uint16_t)run;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int s = 4 * lane + i;  // cdf index s = sum of f[0..s-1]
    if (s <= kNSym) row[s] = (uint16_t)(s == kNSym ? kM : run);
    run += f[i];
  }
}

// ---------------------------------------------------------------------------
// rANS decoding. One warp per chunk; lane l < nl owns symbols l, l+nl, ...
// Round 0 of every iteration decodes each active lane's main symbol; escape
// symbols are followed by bypass rounds (frequency M/2 per bit). After each
// round the lanes whose state fell below 2^16 read one 16-bit word each, in
// ascending lane order (ballot + popc). All loops are bounded by the chunk
// size and the escape-length limit; overruns set kStCorrupt and stop.

// DecChunk (ctx_kernels.cuh): data = nl u32 states then u16 words; count
// symbols; first = index of its first symbol in the output list.

// SWAR compare of the two u16 entries of w against slot (< 2^15): with
// s2 = (slot | 0x8000) in both halves, each half of s2 - w is
// 0x8000 + slot - e, which lies in [0, 0xFFFF] for every entry e <= 2^15,
// so no borrow crosses the halves and bit 15 of a half is set exactly when
// e <= slot. Returns those two bits at positions 0 and 16.
__device__ __forceinline__ uint32_t le2(uint32_t s2, uint32_t w) {
  return ((s2 - w) >> 15) & 0x10001u;
}
// Two consecutive 16-bit words k, k + 1 of a chunk's word stream (0 past the
// end), byte loads so that no alignment is assumed.
__device__ __forceinline__ uint32_t ld_words2(const uint8_t *wp, uint32_t k, uint32_t nwords) {
  uint32_t v = 0;
  if (k < nwords) v = (uint32_t)__ldg(wp + 2 * k) | ((uint32_t)__ldg(wp + 2 * k + 1) << 8);
  if (k + 1 < nwords)
    v |= ((uint32_t)__ldg(wp + 2 * k + 2) << 16) | ((uint32_t)__ldg(wp + 2 * k + 3) << 24);
  return v;
}

// Symbol search: the largest s in [0, 126] with t[s] <= slot, in two levels:
// the table's 16 coarse entries (every 8th, shared memory) give the block
// b = s / 8, one 16-byte load gives its 8 entries. The entries are strictly
// increasing with t[0] = 0, t[127] = M = 2^15 > slot, and all are <= 2^15,
// so the SWAR counts below are exactly that s. Returns s; lo = t[s],
// hi = t[s + 1].
// The table's coarse entries come in registers (c0 = entries 0..7, c1 =
// 8..15, two per word, low half first), loaded one round ahead; the entry
// after block b also comes from them.
__device__ __forceinline__ int cdf_search_r(const uint16_t *__restrict__ row, const uint4 c0,
                                            const uint4 c1, uint32_t slot, uint32_t &lo,
                                            uint32_t &hi) {
  const uint32_t s2 = (slot | 0x8000u) * 0x10001u;
  uint32_t a = le2(s2, c0.x) + le2(s2, c0.y) + le2(s2, c0.z) + le2(s2, c0.w) + le2(s2, c1.x) +
               le2(s2, c1.y) + le2(s2, c1.z) + le2(s2, c1.w);
  const int b = (int)((a & 0xFFFFu) + (a >> 16)) - 1;
  const uint4 f = __ldg(reinterpret_cast<const uint4 *>(row + 8 * b));
  a = le2(s2, f.x) + le2(s2, f.y) + le2(s2, f.z) + le2(s2, f.w);
  const int i = (int)((a & 0xFFFFu) + (a >> 16)) - 1;
  // coarse entry b + 1 (clamped; its low 16 bits are what is used)
  const int bn = min(b + 1, kCoarse - 1), wn = bn >> 1;
  const uint32_t q0 = (wn & 1) ? c0.y : c0.x, q1 = (wn & 1) ? c0.w : c0.z;
  const uint32_t q2 = (wn & 1) ? c1.y : c1.x, q3 = (wn & 1) ? c1.w : c1.z;
  const uint32_t r0 = (wn & 2) ? q1 : q0, r1 = (wn & 2) ? q3 : q2;
  const uint32_t wsel = (wn & 4) ? r1 : r0;
  const uint32_t nxt = (bn & 1) ? (wsel >> 16) : wsel;
  const int wi = i >> 1;
  const uint32_t w0 = (wi & 2) ? ((wi & 1) ? f.w : f.z) : ((wi & 1) ? f.y : f.x);
  const uint32_t w1 = (wi & 2) ? ((wi & 1) ? nxt : f.w) : ((wi & 1) ? f.z : f.y);
  const uint32_t pair = (i & 1) ? __funnelshift_r(w0, w1, 16) : w0;
  lo = pair & 0xFFFFu;
  hi = pair >> 16;
  return 8 * b + i;
}

// Output modes: positions of a four-step subband plane (step >= 0), or a
// linear array (step < 0, out[first + i]).
//
// The block first copies the coarse table bank (64 KB) into shared memory.
// Per round each lane's packed table index was loaded one round earlier;
// the renormalisation words come from a 128-word window that the warp keeps
// in registers (lane l holds words wb + 2l, wb + 2l + 1 in cur and the same
// 64 words later in nxt) and reads with shuffles; the window moves by 64
// words once 64 are consumed, loading the next 64 one shift ahead.
//
// kMix (logistic mixture): every symbol has its own table row in global
// memory (bank = the step's rows, kMixRow entries each, the coarse level in
// the row's last 16), written just before by the mixture head; idx holds
// the centres. The coarse entries of a lane's symbol are loaded two rounds
// ahead, its fine row prefetched into L1 two rounds ahead.
// kRag (ragged batches, Laplace, step >= 0): planes of different sizes on
// one canvas of width w. A chunk's symbols are the step positions of its
// own plane, whose subband width is ext[plane].y >> esh; their packed
// indices sit at the canvas's step positions (the context model runs on the
// canvas) and their values go to canvas rows of stride w.
template <bool kMix, bool kRag>
__global__ void __launch_bounds__(256) k_rans_decode(
    const DecChunk *__restrict__ chunks, int nchunks, const uint16_t *__restrict__ bank,
    const uint16_t *__restrict__ coarse, const uint32_t *__restrict__ idx, int64_t idx_stride,
    int32_t *__restrict__ out, int64_t out_stride, int h, int w, int step,
    uint32_t *status, const int2 *__restrict__ ext, int esh) {
  extern __shared__ uint4 s_coarse4[];
  if constexpr (!kMix) {
    // the coarse level (64 KB) in one asynchronous bulk copy, whatever the
    // block's size; an mbarrier after it counts the bytes
    constexpr uint32_t kBytes = kNTables * kCoarse * 2;
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_coarse4 + kBytes / 16);
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      mbar_expect_tx(bar, kBytes);
      for (uint32_t off = 0; off < kBytes; off += 32768u)
        bulk_load(reinterpret_cast<uint8_t *>(s_coarse4) + off,
                  reinterpret_cast<const uint8_t *>(coarse) + off, min(32768u, kBytes - off),
                  bar);
    }
    __syncthreads();
    // bounded: on expiry the status says so and the block leaves after the
    // copy has had ample time to land
    if (!mbar_wait_drain(bar, 0)) {
      if (threadIdx.x == 0) atomicOr(status, kStTimeout);
      return;
    }
  }
  const uint16_t *s_coarse = reinterpret_cast<const uint16_t *>(s_coarse4);
  const int cw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (cw >= nchunks) return;
  const DecChunk ch = chunks[cw];
  const int nl = ch.lanes;
  if (nl < 1 || nl > 32 || ch.nbytes < 4u * nl || ((ch.nbytes - 4u * nl) & 1u)) {
    if (lane == 0) atomicOr(status, kStCorrupt);
    return;
  }
  const uint32_t nwords = (ch.nbytes - 4u * nl) >> 1;
  const uint8_t *base = ch.data;
  uint32_t x = kRansL;
  if (lane < nl) {
    const uint8_t *sp = base + 4 * lane;
    x = (uint32_t)sp[0] | ((uint32_t)sp[1] << 8) | ((uint32_t)sp[2] << 16) |
        ((uint32_t)sp[3] << 24);
  }
  const uint8_t *wp = base + 4 * nl;
  uint32_t wb = 0;
  uint32_t wcur = ld_words2(wp, 2 * lane, nwords), wnxt = ld_words2(wp, 64 + 2 * lane, nwords);
  uint32_t ptr = 0;
  bool bad = false;
  const uint32_t lt = (1u << lane) - 1u;
  // word k of the stream (k - wb in [0, 128) for every calling lane)
  auto word = [&](uint32_t k) -> uint32_t {
    const uint32_t r = k - wb;
    const int src = (int)((r & 63u) >> 1);
    const uint32_t a = __shfl_sync(0xffffffffu, wcur, src);
    const uint32_t b = __shfl_sync(0xffffffffu, wnxt, src);
    const uint32_t v = r < 64u ? a : b;
    return (r & 1u) ? (v >> 16) : (v & 0xFFFFu);
  };
  auto advance = [&](uint32_t n) {
    ptr += n;
    if (ptr - wb >= 64u) {
      wcur = wnxt;
      wnxt = ld_words2(wp, wb + 128 + 2 * lane, nwords);
      wb += 64;
    }
  };
  const uint32_t *idxp = idx + (int64_t)ch.plane * idx_stride;
  int32_t *outp = out + (int64_t)ch.plane * out_stride;
  const int count = (int)ch.count;
  if (kMix && count == 0) {  // chunk layouts hold no empty chunks
    if (lane == 0) atomicOr(status, kStCorrupt);
    return;
  }
  const int niter = (count + nl - 1) / nl;
  // output position of symbol q = first + p (step layout): row pair y2,
  // index r within the pair, advanced by nl per iteration
  int ae = 0, ao = 0, ne = 1, pair = 1, y2 = 0, rr = 0, neC = 0, pairC = 0;
  if (step >= 0) {
    ae = step_phase(step, 0); ao = step_phase(step, 1);
    const int wq = kRag ? (ext[ch.plane].y >> esh) : w;
    ne = row_count(wq, ae);
    pair = ne + row_count(wq, ao);
    if (kRag) {
      neC = row_count(w, ae);
      pairC = neC + row_count(w, ao);
    }
    if (pair == 0 || wq > w) {  // a step without positions has no chunks
      if (lane == 0) atomicOr(status, kStCorrupt);
      return;
    }
    const int q0 = (int)ch.first + lane;
    y2 = q0 / pair; rr = q0 - y2 * pair;
  }
  // idx element of the chunk's symbol i: its step index, or (kRag) the
  // canvas step index of its position
  auto ix = [&](int i) -> int64_t {
    const int q = (int)ch.first + i;
    if constexpr (kRag) {
      const int a2 = q / pair, r = q - a2 * pair;
      return (int64_t)a2 * pairC + (r < ne ? r : neC + (r - ne));
    } else {
      return q;
    }
  };
  // packed indices of this lane's next two symbols and the coarse row of
  // the next one, fetched a round ahead so that neither load is on the
  // round's dependent chain (every unpacked index is a valid table)
  uint32_t pk_a = (lane < nl && lane < count) ? __ldg(idxp + ix(lane)) : 0u;
  uint32_t pk_b = (lane < nl && lane + nl < count) ? __ldg(idxp + ix(lane + nl)) : 0u;
  uint4 ca0, ca1, cb0, cb1;
  // kMix: row of the chunk's symbol i (inactive lanes use the first one)
  const uint16_t *mrows = bank + ((int64_t)ch.plane * idx_stride + ch.first) * kMixRow;
  auto mix_row = [&](int i) { return mrows + (int64_t)(i < count ? i : 0) * kMixRow; };
  if constexpr (kMix) {
    const uint4 *ra = reinterpret_cast<const uint4 *>(mix_row(lane) + kNSym + 1);
    const uint4 *rb = reinterpret_cast<const uint4 *>(mix_row(lane + nl) + kNSym + 1);
    ca0 = __ldg(ra); ca1 = __ldg(ra + 1);
    cb0 = __ldg(rb); cb1 = __ldg(rb + 1);
  } else {
    int c, t;
    unpack_index(pk_a, c, t);
    const uint4 *cr = reinterpret_cast<const uint4 *>(s_coarse + t * kCoarse);
    ca0 = cr[0]; ca1 = cr[1];
  }
  for (int it = 0; it < niter; ++it) {
    const int p = it * nl + lane;
    const bool active = lane < nl && p < count;
    const uint32_t pk = pk_a;
    const uint4 c0 = ca0, c1 = ca1;
    if constexpr (kMix) {
      ca0 = cb0; ca1 = cb1;
      const uint16_t *frow = mix_row(p + 2 * nl);
      const uint4 *cr = reinterpret_cast<const uint4 *>(frow + kNSym + 1);
      cb0 = __ldg(cr); cb1 = __ldg(cr + 1);
      asm volatile("prefetch.global.L1 [%0];" ::"l"(frow));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(frow + 64));
    } else {
      int c, t;
      unpack_index(pk_b, c, t);
      const uint4 *cr = reinterpret_cast<const uint4 *>(s_coarse + t * kCoarse);
      ca0 = cr[0]; ca1 = cr[1];
      // and its fine level (256 bytes, two L1 lines) into L1, so that next
      // round's dependent 16-byte load hits there
      const uint16_t *frow = bank + (size_t)t * (kNSym + 1);
      asm volatile("prefetch.global.L1 [%0];" ::"l"(frow));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(frow + 64));
    }
    pk_a = pk_b;
    pk_b = (active && p + 2 * nl < count) ? __ldg(idxp + ix(p + 2 * nl)) : 0u;
    // every lane runs the search (inactive lanes on a valid table, their
    // state kept), so the round has no branch around it
    int ctr;
    const uint16_t *trow;
    if constexpr (kMix) {
      ctr = (int)pk;
      trow = mix_row(active ? p : 0);
    } else {
      int tid;
      unpack_index(pk, ctr, tid);
      trow = bank + (size_t)tid * (kNSym + 1);
    }
    const uint32_t slot = x & (kM - 1);
    uint32_t lo, hi;
    const int s = cdf_search_r(trow, c0, c1, slot, lo, hi);
    {
      const uint32_t xn = (hi - lo) * (x >> kLogM) + slot - lo;
      x = active ? xn : x;
      const bool need = active && x < kRansL;
      const uint32_t m = __ballot_sync(0xffffffffu, need);
      const uint32_t k = ptr + __popc(m & lt);
      const uint32_t wv = word(need ? k : ptr);
      bad = bad || (need && k >= nwords);
      x = need ? ((x << 16) | (k < nwords ? wv : 0u)) : x;
      advance(__popc(m));
    }
    // escapes: phase 0 counts ones up to a zero, phase 1 reads k bits
    bool pend = active && (s == 0 || s == kNSym - 1);
    int phase = 0, kcnt = 0;
    uint32_t v = 0;
    if (__builtin_expect(__any_sync(0xffffffffu, pend), 0))
    for (int rnd = 0; rnd < 2 * kMaxEscBits + 2; ++rnd) {
      if (!__any_sync(0xffffffffu, pend)) break;
      if (pend) {
        const uint32_t slot = x & (kM - 1);
        const uint32_t bit = slot >> (kLogM - 1);
        x = (kM >> 1) * (x >> kLogM) + (slot & ((kM >> 1) - 1));
        if (phase == 0) {
          if (bit) { if (++kcnt > kMaxEscBits) { bad = true; } }
          else { phase = 1; v = 1; }
        } else {
          v = (v << 1) | bit;
          --kcnt;
        }
      }
      const bool need = pend && x < kRansL;
      const uint32_t m = __ballot_sync(0xffffffffu, need);
      if (m) {
        const uint32_t k = ptr + __popc(m & lt);
        const uint32_t wv = word(need ? k : ptr);
        if (need) {
          if (k >= nwords) bad = true;
          x = (x << 16) | (k < nwords ? wv : 0u);
        }
        advance(__popc(m));
      }
      if (pend && ((phase == 1 && kcnt == 0) || bad)) pend = false;
    }
    if (pend) bad = true;
    if (active) {
      int r;
      if (s == 0) r = -(int)(v - 1) - kT - 1;
      else if (s == kNSym - 1) r = (int)(v - 1) + kT + 1;
      else r = s - kT - 1;
      const int val = ctr + r;
      if (step >= 0) {
        const int yy = rr < ne ? 2 * y2 : 2 * y2 + 1;
        const int xx = rr < ne ? ae + 4 * rr : ao + 4 * (rr - ne);
        outp[(int64_t)yy * w + xx] = val;
      } else {
        outp[ch.first + p] = val;
      }
    }
    if (step >= 0) {
      rr += nl;
      if (nl <= pair) {
        const bool wrap = rr >= pair;
        rr -= wrap ? pair : 0;
        y2 += wrap ? 1 : 0;
      } else {
        while (rr >= pair) { rr -= pair; ++y2; }
      }
    }
    // every loop is bounded, so a corrupt chunk only has to stop early
    // eventually: vote every 32 iterations
    if ((it & 31) == 31 && __any_sync(0xffffffffu, bad)) break;
  }
  if (lane < nl && x != kRansL) bad = true;
  if (lane == 0 && ptr != nwords) bad = true;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStCorrupt);
}

// ---------------------------------------------------------------------------
// rANS encoding (reverse of the decoder). One warp per chunk; iterations,
// rounds and lanes run in descending order; each emitted word is written at
// a decreasing address of the chunk's scratch region, so the words read
// forward from the lowest written address are in decoder order.

// EncChunk (ctx_kernels.cuh): the chunk's symbols are idx[sym_base + i] /
// vals[sym_base + i]; scratch_end = word index one past its scratch region.

__device__ __forceinline__ void esc_code(int r, int &s, uint32_t &v, int &k) {
  if (r >= -kT && r <= kT) { s = r + kT + 1; v = 0; k = -1; return; }
  uint32_t e = (r < -kT) ? (uint32_t)(-r - kT - 1) : (uint32_t)(r - kT - 1);
  s = (r < -kT) ? 0 : kNSym - 1;
  v = e + 1;
  k = 31 - __clz(v);
}

// ops of a symbol: 1 main + (2k + 1) bypass bits for an escape
// (mix: idx holds the centres)
__global__ void k_rans_count_ops(const EncChunk *__restrict__ chunks, int nchunks,
                                 const uint32_t *__restrict__ idx,
                                 const int32_t *__restrict__ vals,
                                 uint32_t *__restrict__ ops, int mix) {
  const int cw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (cw >= nchunks) return;
  EncChunk ch = chunks[cw];
  uint32_t tot = 0;
  for (uint32_t i = lane; i < ch.count; i += 32) {
    const int64_t q = (int64_t)ch.sym_base + i;
    int ctr, tid;
    if (mix) ctr = (int)idx[q];
    else unpack_index(idx[q], ctr, tid);
    int s, k;
    uint32_t v;
    esc_code(vals[q] - ctr, s, v, k);
    tot += 1 + (k >= 0 ? 2 * k + 1 : 0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if (lane == 0) ops[cw] = tot;
}

__global__ void k_rans_encode(const EncChunk *__restrict__ chunks, int nchunks,
                              const uint16_t *__restrict__ bank,
                              const uint32_t *__restrict__ idx,
                              const int32_t *__restrict__ vals,
                              uint16_t *__restrict__ scratch,
                              uint32_t *__restrict__ states_out,  // 32 per chunk
                              uint32_t *__restrict__ nwords_out, uint32_t *status,
                              const uint32_t *__restrict__ cf) {
  const int cw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (cw >= nchunks) return;
  const EncChunk ch = chunks[cw];
  const int nl = ch.lanes;
  uint32_t x = kRansL;
  uint64_t wpos = ch.scratch_end;
  const uint32_t gt = ~((2u << lane) - 1u);  // lanes above me
  const int niter = (ch.count + nl - 1) / nl;
  bool bad = false;
  for (int it = niter - 1; it >= 0; --it) {
    const int p = it * nl + lane;
    const bool active = lane < nl && p < (int)ch.count;
    int s = 0, k = -1;
    uint32_t v = 0, c0 = 0, f0 = 1;
    if (active) {
      const int64_t q = (int64_t)ch.sym_base + p;
      int ctr, tid;
      if (cf) {
        // logistic mixture: the symbol's own (cdf, frequency), centre in idx
        ctr = (int)idx[q];
        esc_code(vals[q] - ctr, s, v, k);
        c0 = cf[q] & 0xFFFFu;
        f0 = cf[q] >> 16;
      } else {
        unpack_index(idx[q], ctr, tid);
        esc_code(vals[q] - ctr, s, v, k);
        const uint16_t *t = bank + (size_t)tid * (kNSym + 1);
        c0 = t[s];
        f0 = (uint32_t)t[s + 1] - c0;
      }
      if (k > kMaxEscBits) bad = true;
    }
    const int nops = active ? 1 + (k >= 0 ? 2 * k + 1 : 0) : 0;
    int rounds = nops;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(0xffffffffu, rounds, o));
    for (int rnd = rounds - 1; rnd >= 0; --rnd) {
      const bool has = rnd < nops;
      uint32_t c = c0, f = f0;
      if (has && rnd > 0) {
        int b = rnd - 1;          // bypass bit index in decode order
        uint32_t bit;
        if (b < k) bit = 1;
        else if (b == k) bit = 0;
        else bit = (v >> (2 * k - b)) & 1u;
        c = bit * (kM >> 1);
        f = kM >> 1;
      }
      const bool emit = has && x >= (f << 17);
      const uint32_t m = __ballot_sync(0xffffffffu, emit);
      if (emit) {
        uint64_t pos = wpos - 1 - __popc(m & gt);
        scratch[pos] = (uint16_t)(x & 0xFFFFu);
        x >>= 16;
      }
      wpos -= __popc(m);
      if (has) x = (x / f) * kM + (x % f) + c;
    }
  }
  if (lane < nl) states_out[(size_t)cw * 32 + lane] = x;
  if (lane == 0) nwords_out[cw] = (uint32_t)(ch.scratch_end - wpos);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStRange);
}

// Copy encoded chunks (states + words) into the packed payload.
__global__ void k_rans_pack(const EncChunk *__restrict__ chunks, int nchunks,
                            const uint16_t *__restrict__ scratch,
                            const uint32_t *__restrict__ states,
                            const uint32_t *__restrict__ nwords,
                            const uint64_t *__restrict__ out_off,
                            uint8_t *__restrict__ payload) {
  const int cw = blockIdx.x;
  if (cw >= nchunks) return;
  const EncChunk ch = chunks[cw];
  const int nl = ch.lanes;
  uint8_t *dst = payload + out_off[cw];
  for (int i = threadIdx.x; i < 4 * nl; i += blockDim.x) {
    uint32_t st = states[(size_t)cw * 32 + i / 4];
    dst[i] = (uint8_t)(st >> (8 * (i & 3)));
  }
  const uint32_t nw = nwords[cw];
  const uint16_t *src = scratch + (ch.scratch_end - nw);
  uint8_t *dw = dst + 4 * nl;
  for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) {
    uint16_t v = src[i];
    dw[2 * i] = (uint8_t)(v & 0xFF);
    dw[2 * i + 1] = (uint8_t)(v >> 8);
  }
}

// Entropy-parameter index decision over arrays (stage API).
__global__ void k_pack_index(const float *__restrict__ mu, const float *__restrict__ rho_or_sigma,
                             int64_t n, int is_sigma, uint32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float m = mu[i], s = rho_or_sigma[i];
  if (is_sigma) {
    // sigma given directly: bypass the softplus by mapping through rho = s
    // only for the bin computation
    float t = rintf(__fmul_rn(m, 16.f));
    t = fminf(fmaxf(t, -8388608.f), 8388608.f);
    int j = (__float_as_int(s) - 0x3E000000) >> 20;
    j = min(max(j, 0), kNJ - 1);
    idx[i] = ((uint32_t)((int)t + (1 << 23)) << 7) | (uint32_t)j;
  } else {
    idx[i] = pack_index(m, s);
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
void launch_cdf_bank(uint16_t *bank, uint16_t *coarse, cudaStream_t st) {
  k_cdf_bank<<<kNTables * 32 / 256, 256, 0, st>>>(bank, coarse);
}
void launch_rans_decode(const DecChunk *chunks, int nchunks, const uint16_t *bank,
                        const uint16_t *coarse, const uint32_t *idx, int64_t idx_stride,
                        int32_t *out, int64_t out_stride, int h, int w, int step,
                        uint32_t *status, cudaStream_t st, bool mix, const int2 *ext,
                        int esh) {
  if (nchunks <= 0) return;
  const int nsm = sm_count();
  if (mix) {
    int wpb = 8;
    while (wpb > 1 && (nchunks + wpb - 1) / wpb < nsm) wpb >>= 1;
    k_rans_decode<true, false><<<(nchunks + wpb - 1) / wpb, 32 * wpb, 0, st>>>(
        chunks, nchunks, bank, nullptr, idx, idx_stride, out, out_stride, h, w, step, status,
        nullptr, 0);
    return;
  }
  constexpr int smem = kNTables * kCoarse * 2 + 16;   // coarse level + mbarrier
  static std::atomic<uint64_t> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_rans_decode<false, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_rans_decode<false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  // one warp per chunk; with few chunks, fewer warps per block so that the
  // chunks spread over the SMs (one warp per scheduler)
  int wpb = 8;
  while (wpb > 1 && (nchunks + wpb - 1) / wpb < nsm) wpb >>= 1;
  if (ext && step >= 0)
    k_rans_decode<false, true><<<(nchunks + wpb - 1) / wpb, 32 * wpb, smem, st>>>(
        chunks, nchunks, bank, coarse, idx, idx_stride, out, out_stride, h, w, step, status,
        ext, esh);
  else
    k_rans_decode<false, false><<<(nchunks + wpb - 1) / wpb, 32 * wpb, smem, st>>>(
        chunks, nchunks, bank, coarse, idx, idx_stride, out, out_stride, h, w, step, status,
        nullptr, 0);
}
void launch_rans_count_ops(const EncChunk *chunks, int nchunks, const uint32_t *idx,
                           const int32_t *vals, uint32_t *ops, cudaStream_t st, bool mix) {
  if (nchunks <= 0) return;
  k_rans_count_ops<<<(nchunks + 3) / 4, 128, 0, st>>>(chunks, nchunks, idx, vals, ops,
                                                      mix ? 1 : 0);
}
void launch_rans_encode(const EncChunk *chunks, int nchunks, const uint16_t *bank,
                        const uint32_t *idx, const int32_t *vals, uint16_t *scratch,
                        uint32_t *states, uint32_t *nwords, uint32_t *status,
                        cudaStream_t st, const uint32_t *cf) {
  if (nchunks <= 0) return;
  k_rans_encode<<<(nchunks + 3) / 4, 128, 0, st>>>(chunks, nchunks, bank, idx, vals, scratch,
                                                   states, nwords, status, cf);
}
void launch_rans_pack(const EncChunk *chunks, int nchunks, const uint16_t *scratch,
                      const uint32_t *states, const uint32_t *nwords,
                      const uint64_t *out_off, uint8_t *payload, cudaStream_t st) {
  if (nchunks <= 0) return;
  k_rans_pack<<<nchunks, 256, 0, st>>>(chunks, nchunks, scratch, states, nwords, out_off,
                                       payload);
}
void launch_pack_index(const float *mu, const float *s, int64_t n, int is_sigma,
                       uint32_t *idx, cudaStream_t st) {
  if (n <= 0) return;
  k_pack_index<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mu, s, n, is_sigma, idx);
}

}  // namespace pw
