// Decode server: continuous batching of decode requests of mixed sizes.
//
// Requests (host bitstreams) enter a queue. Worker lanes, each with its own
// CUDA stream and workspace cache, repeatedly take the oldest queued request
// together with queued requests of the same format (channels, levels, bit
// depth, coder layout; up to max_batch) whose sizes are close enough: a
// request joins while the batch's canvas (the largest padded size) times
// its image count stays within kCanvasWaste times the images' own padded
// area. The batch is decoded in one call - a ragged batch when the sizes
// differ, whose every launch covers all its images. (Logistic-mixture
// models batch identical sizes only.) A batch is admitted
// only when the device memory it needs (its workspace estimate) fits in the
// HBM budget next to what the other lanes hold, so requests that arrive while
// others are on the GPU start as soon as a lane and memory free up, and the
// lanes' kernels overlap on the device. Decoding is deterministic and every
// image of a batch is computed independently, so a result is identical
// whether the request was decoded alone or in a mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "codec.h"

using Clock = std::chrono::steady_clock;

namespace pw {

struct Req {
  uint64_t ticket = 0;
  std::vector<uint8_t> bs;
  std::string key;           // geometry (size and format)
  std::string fkey;          // format only (ragged batches share it)
  Geometry g;
  int64_t need = 0;          // workspace bytes of a batch of one (estimate)
  Clock::time_point t_submit, t_done;
  int status = PW_OK;
  std::string error;         // error text of a failed decode
  bool done = false;
  std::vector<uint8_t> out;  // decoded image (host, packed HWC)
};

}  // namespace pw

struct pw_server {
  pw_ctx *ctx = nullptr;
  pw::Model *m = nullptr;
  int64_t budget = 0;
  int max_batch = 8;
  std::vector<pw_ctx *> lanes;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> threads;
  std::vector<int64_t> lane_bytes;
  std::vector<std::string> lane_key;
  int64_t held = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<pw::Req *> queue;
  std::map<uint64_t, pw::Req *> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  // statistics
  std::vector<double> lat_ms;
  uint64_t submitted = 0, completed = 0, failed = 0, rejected = 0, batches = 0;
  double pixels = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace pw {

static std::string fmt_key(const Geometry &g) {
  char b[160];
  snprintf(b, sizeof(b), "%d:%d:%d:%d:%d:%d:%d:%d:%d", g.nc, g.levels, g.colour, g.bitdepth,
           g.lossless, g.ll_ar, g.chunk, g.balanced, g.lane_shift);
  return b;
}
static std::string req_key(const Geometry &g) {
  return std::to_string(g.H) + "x" + std::to_string(g.W) + ":" + fmt_key(g);
}

// A ragged batch's canvas area may exceed its images' own padded area by at
// most this factor (the work spent on the canvas outside the images).
constexpr double kCanvasWaste = 1.5;

// Geometry of the canvas of a batch: the largest padded size (the first
// request's geometry when all sizes are equal).
static Geometry canvas_of(const std::vector<Req *> &batch) {
  const Geometry &g0 = batch[0]->g;
  int Hc = 0, Wc = 0;
  bool same = true;
  for (Req *q : batch) {
    Hc = std::max(Hc, q->g.Hp);
    Wc = std::max(Wc, q->g.Wp);
    same = same && q->g.H == g0.H && q->g.W == g0.W;
  }
  if (same) return g0;
  Geometry gc;
  gc.build(Hc, Wc, g0.nc, g0.levels, g0.colour, g0.bitdepth, g0.lossless, g0.ll_ar, g0.chunk,
           g0.balanced, g0.lane_shift);
  return gc;
}

// The oldest queued request and the queued requests that batch with it.
static std::vector<Req *> form_batch(const std::deque<Req *> &queue, int max_batch, bool ragged) {
  Req *r0 = queue.front();
  std::vector<Req *> batch{r0};
  int Hc = r0->g.Hp, Wc = r0->g.Wp;
  double area = (double)r0->g.Hp * r0->g.Wp;
  for (Req *q : queue) {
    if ((int)batch.size() >= max_batch) break;
    if (q == r0) continue;
    if (!ragged) {
      if (q->key == r0->key) batch.push_back(q);
      continue;
    }
    if (q->fkey != r0->fkey) continue;
    const int h = std::max(Hc, q->g.Hp), w = std::max(Wc, q->g.Wp);
    const double a = area + (double)q->g.Hp * q->g.Wp;
    if ((double)(batch.size() + 1) * h * w > kCanvasWaste * a) continue;
    batch.push_back(q);
    Hc = h;
    Wc = w;
    area = a;
  }
  return batch;
}

static void lane_main(pw_server *s, int li) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  // Give this lane's workspace back (called with the lock held).
  auto release_own = [&]() {
    if (!s->lane_bytes[li]) return;
    lk.unlock();
    drop_plans(s->lanes[li]);
    lk.lock();
    s->held -= s->lane_bytes[li];
    s->lane_bytes[li] = 0;
    s->lane_key[li].clear();
    s->cv_done.notify_all();
  };
  const int prec = s->lanes[li]->precision;
  while (!s->stop) {
    if (s->queue.empty()) {
      release_own();  // idle: the memory goes back to the budget
      s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    std::vector<Req *> batch = form_batch(s->queue, s->max_batch, !s->m->mix);
    // the largest batch whose workspace fits next to the other lanes'
    const int64_t others = s->held - s->lane_bytes[li];
    int64_t need = 0;
    Geometry gc;
    for (;;) {
      gc = canvas_of(batch);
      need = Workspace::estimate(gc, (int)batch.size() * gc.nc, s->m->C, false, prec, s->m->mix);
      if (others + need <= s->budget || batch.size() == 1) break;
      batch.pop_back();
    }
    if (others + need > s->budget && others > 0) {
      // wait for another lane to finish; free this lane's memory meanwhile so
      // that two waiting lanes cannot block each other
      release_own();
      s->cv_done.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    for (Req *q : batch) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), q));
    // a context caches one workspace per (canvas geometry, batch size): keep
    // it only when both repeat
    const std::string lkey = req_key(gc) + "#" + std::to_string(batch.size());
    const bool same = s->lane_key[li] == lkey;
    s->held = others + need;
    s->lane_bytes[li] = need;
    s->lane_key[li] = lkey;
    lk.unlock();
    if (!same) drop_plans(s->lanes[li]);
    const int B = (int)batch.size();
    std::vector<const uint8_t *> ptrs(B);
    std::vector<size_t> lens(B);
    std::vector<pw_image> outs(B);
    for (int b = 0; b < B; ++b) {
      Req *q = batch[b];
      const Geometry &g = q->g;
      const int bps = g.bitdepth > 8 ? 2 : 1;
      ptrs[b] = q->bs.data();
      lens[b] = q->bs.size();
      q->out.assign((size_t)g.H * g.W * g.nc * bps, 0);
      outs[b] = pw_image{g.W, g.H, g.nc, g.bitdepth, 0, 0, q->out.data(), 0};
    }
    std::vector<int> st(B, decode_batch(s->lanes[li], *s->m, B, ptrs.data(), lens.data(), 0,
                                        outs.data()));
    std::vector<std::string> err(B, st[0] == PW_OK ? std::string() : pw_last_error());
    if (st[0] != PW_OK && B > 1) {
      // isolate the failing request(s): decode each one alone
      for (int b = 0; b < B; ++b) {
        st[b] = decode_batch(s->lanes[li], *s->m, 1, &ptrs[b], &lens[b], 0, &outs[b]);
        err[b] = st[b] == PW_OK ? std::string() : pw_last_error();
      }
    }
    lk.lock();
    const auto now = Clock::now();
    ++s->batches;
    for (int b = 0; b < B; ++b) {
      Req *q = batch[b];
      q->status = st[b];
      q->error = err[b];
      q->done = true;
      q->t_done = now;
      s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - q->t_submit).count());
      if (st[b] == PW_OK) {
        ++s->completed;
        s->pixels += (double)q->g.H * q->g.W;
      } else {
        ++s->failed;
      }
    }
    s->t_last = now;
    s->cv_done.notify_all();
  }
}

}  // namespace pw

using namespace pw;

extern "C" {

int pw_server_create(pw_ctx *ctx, const pw_model *m, size_t hbm_budget, int lanes, int max_batch,
                     pw_server **out) {
  if (!ctx || !m || !out || lanes < 1 || lanes > 16 || max_batch < 1) return PW_EINVAL;
  pw_server *s = new pw_server();
  s->ctx = ctx;
  s->m = &const_cast<pw_model *>(m)->m;
  s->budget = (int64_t)hbm_budget;
  s->max_batch = max_batch;
  for (int i = 0; i < lanes; ++i) {
    cudaStream_t st = nullptr;
    pw_ctx *lc = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        pw_ctx_create(ctx->device, st, ctx->precision, &lc) != PW_OK) {
      if (st) cudaStreamDestroy(st);
      pw_server_destroy(s);
      set_last_error("server lane creation failed");
      return PW_ECUDA;
    }
    s->streams.push_back(st);
    s->lanes.push_back(lc);
    s->lane_bytes.push_back(0);
    s->lane_key.push_back("");
  }
  for (int i = 0; i < lanes; ++i) s->threads.emplace_back(lane_main, s, i);
  *out = s;
  return PW_OK;
}

void pw_server_destroy(pw_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->threads) t.join();
  for (pw_ctx *c : s->lanes) pw_ctx_destroy(c);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (auto &kv : s->reqs) delete kv.second;  // every queued request is in reqs
  delete s;
}

int pw_server_submit(pw_server *s, const uint8_t *bs, size_t n, uint64_t *ticket) {
  if (!s || !bs || !ticket) return PW_EINVAL;
  Req *r = new Req();
  int st = stream_geometry(s->ctx, *s->m, bs, n, r->g);
  if (st != PW_OK) {
    delete r;
    return st;
  }
  r->key = req_key(r->g);
  r->fkey = fmt_key(r->g);
  r->need = Workspace::estimate(r->g, r->g.nc, s->m->C, false, s->ctx->precision, s->m->mix);
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->need > s->budget || s->queue.size() >= 4096) {
    ++s->rejected;
    delete r;
    set_last_error("request does not fit the server's HBM budget or queue");
    return PW_EAGAIN;
  }
  r->bs.assign(bs, bs + n);
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  if (!s->have_first) { s->t_first = r->t_submit; s->have_first = true; }
  s->queue.push_back(r);
  s->reqs[r->ticket] = r;
  ++s->submitted;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return PW_OK;
}

int pw_server_poll(pw_server *s, uint64_t ticket, pw_image *out, int timeout_ms) {
  if (!s || !out) return PW_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) { set_last_error("unknown ticket"); return PW_EINVAL; }
  Req *r = it->second;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (!r->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
      return timeout_ms == 0 ? PW_EAGAIN : PW_ETIMEOUT;
  }
  const Geometry &g = r->g;
  const int bps = g.bitdepth > 8 ? 2 : 1;
  int st = r->status;
  if (st != PW_OK) set_last_error(r->error);
  if (st == PW_OK) {
    if (out->width != g.W || out->height != g.H || out->channels != g.nc || !out->data ||
        (out->bitdepth > 8 ? 2 : 1) != bps) {
      set_last_error("output image does not match the request");
      return PW_EINVAL;
    }
    const int64_t row = (int64_t)g.W * g.nc * bps;
    const int64_t rs = out->stride_bytes ? out->stride_bytes : row;
    if (cudaMemcpy2D(out->data, rs, r->out.data(), row, row, g.H,
                     out->is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost) !=
        cudaSuccess) {
      set_last_error("copy of the result failed");
      st = PW_ECUDA;
    }
  }
  s->reqs.erase(it);
  delete r;
  return st;
}

int pw_decode_footprint(pw_ctx *ctx, const pw_model *m, const uint8_t *bs, size_t n, int count,
                        uint64_t *bytes) {
  if (!ctx || !m || !bs || !bytes || count < 1) return PW_EINVAL;
  Geometry g;
  const int st = stream_geometry(ctx, m->m, bs, n, g);
  if (st != PW_OK) return st;
  *bytes = (uint64_t)Workspace::estimate(g, count * g.nc, m->m.C, false, ctx->precision,
                                         m->m.mix);
  return PW_OK;
}

int pw_server_stats(pw_server *s, pw_stats *o) {
  if (!s || !o) return PW_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(o, 0, sizeof(*o));
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->rejected = s->rejected;
  o->queued = s->queue.size();
  o->batches = s->batches;
  o->held_bytes = (uint64_t)s->held;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const double idx = p * (double)(v.size() - 1);
      const size_t i0 = (size_t)idx;
      const size_t i1 = std::min(v.size() - 1, i0 + 1);
      return v[i0] + (v[i1] - v[i0]) * (idx - (double)i0);
    };
    o->p50_ms = pct(0.50);
    o->p99_ms = pct(0.99);
  }
  if (s->have_first && s->completed) {
    const double sec = std::chrono::duration<double>(s->t_last - s->t_first).count();
    o->mpix_per_s = sec > 0 ? s->pixels / sec / 1e6 : 0.0;
  }
  return PW_OK;
}

}  // extern "C"
