// liblrvol frame server: continuous batching of frame requests over volumes
// that stay resident on the device.  Requests queue in FIFO order per size
// tier; each call
// of lrvol_server_progress retires frames whose work has finished (one event
// query per busy slot, never a wait) and admits waiting requests while a slot
// stream is free and the output arena has room, so the frames of several
// requests run concurrently on the GPU.  Every frame runs the same kernels as
// lrvol_render with statistics counters of its own slot.
#include <chrono>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <unordered_map>
#include <vector>

#include "lrvol_internal.h"

using namespace lrvol;

// ----------------------------------------------------------------------------
// arena bookkeeping: first fit over a map of free blocks, coalesced on free
// ----------------------------------------------------------------------------
struct lrvol_arena_s {
  int64_t size = 0, align = 256;
  std::map<int64_t, int64_t> free_blocks;     // offset -> size
  std::unordered_map<int64_t, int64_t> used;  // offset -> size
  int64_t in_use = 0;

  int64_t round(int64_t bytes) const { return ((bytes < 1 ? 1 : bytes) + align - 1) & ~(align - 1); }

  int64_t alloc(int64_t bytes) {
    const int64_t need = round(bytes);
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < need) continue;
      const int64_t off = it->first, rest = it->second - need;
      free_blocks.erase(it);
      if (rest > 0) free_blocks[off + need] = rest;
      used[off] = need;
      in_use += need;
      return off;
    }
    return -1;
  }

  bool release(int64_t off) {
    auto u = used.find(off);
    if (u == used.end()) return false;
    int64_t sz = u->second;
    used.erase(u);
    in_use -= sz;
    auto next = free_blocks.lower_bound(off);
    if (next != free_blocks.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        off = prev->first;
        sz += prev->second;
        free_blocks.erase(prev);
      }
    }
    if (next != free_blocks.end() && off + sz == next->first) {
      sz += next->second;
      free_blocks.erase(next);
    }
    free_blocks[off] = sz;
    return true;
  }

  int64_t largest_free() const {
    int64_t m = 0;
    for (const auto &f : free_blocks) m = f.second > m ? f.second : m;
    return m;
  }
};

namespace {

bool init_arena(lrvol_arena_s *a, int64_t bytes, int64_t align) {
  if (bytes < 1 || align < 1 || (align & (align - 1))) return false;
  a->size = bytes;
  a->align = align;
  a->free_blocks.clear();
  a->used.clear();
  a->in_use = 0;
  a->free_blocks[0] = bytes;
  return true;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr int kSlotScratchBytes = 128;  // kNumCounters counters, then the status word at byte 64
static_assert(kNumCounters * 8 <= 64, "slot scratch layout");

constexpr int kTiers = 3;  // stream priority tiers per slot: small, medium, large frames

struct Request {
  int64_t ticket = 0;
  lrvol_s *vol = nullptr;
  lrvol_camera cam;
  lrvol_tf tf;
  lrvol_step step;
  float *host_out = nullptr;
  bool learned_auto = false;
  int tier = kTiers - 1;  // stream priority tier the frame is launched at
  int32_t state = LRVOL_REQ_QUEUED, status = LRVOL_OK;
  int slot = -1;
  int64_t image_bytes = 0, bytes = 0, off = -1;
  double t_submit = 0, t_admit = 0, t_done = 0;
  float device_ms = 0, dev_start_ms = 0, dev_end_ms = 0;
  int64_t samples = 0, lookups = 0, rays = 0;
};

struct Slot {
  cudaStream_t stream[kTiers] = {nullptr, nullptr, nullptr};  // tier 0 has the highest priority
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  unsigned char *d_scratch = nullptr;  // kSlotScratchBytes
  unsigned char *h_scratch = nullptr;  // pinned mirror
  int64_t ticket = -1;
};

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

}  // namespace

struct lrvol_server_s {
  int device = 0;
  std::vector<Slot> slots;
  unsigned char *d_arena = nullptr;
  unsigned char *d_scratch = nullptr;
  unsigned char *h_scratch = nullptr;
  cudaEvent_t base = nullptr;
  lrvol_arena_s arena;
  std::deque<int64_t> queue[kTiers];  // FIFO per tier (one tier while priorities are off)
  std::deque<int64_t> finished;  // retired since the last lrvol_server_poll
  std::unordered_map<int64_t, Request> req;
  int64_t next_ticket = 1;
  int64_t submitted = 0, done = 0, failed = 0, high_water = 0;
  int running = 0, max_running = 0;
  int running_tier[kTiers] = {0, 0, 0};
  const uint16_t *packed = nullptr;
  float ymin = 0.f, ymax = 0.f;
  int64_t priority_pixels = 0;  // tier 0 up to this many pixels, tier 1 up to 4 times as many, else tier 2
  int large_cap = 0;            // most frames of the last tier in flight (0: slots - max(1, slots/4))
};

namespace {

void free_server(lrvol_server_s *s) {
  for (auto &sl : s->slots) {
    for (cudaStream_t st : sl.stream)
      if (st) cudaStreamSynchronize(st);
    if (sl.ev0) cudaEventDestroy(sl.ev0);
    if (sl.ev1) cudaEventDestroy(sl.ev1);
    for (cudaStream_t st : sl.stream)
      if (st) cudaStreamDestroy(st);
  }
  if (s->base) cudaEventDestroy(s->base);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->d_scratch) cudaFree(s->d_scratch);
  if (s->h_scratch) cudaFreeHost(s->h_scratch);
  delete s;
}

// Launch the admitted request r on slot k: clear the slot's counters, then
// [learned: features, network], render, counters and (optionally) the image
// to the host, bracketed by the slot's two events.
int launch_request(lrvol_server_s *s, Request &r, int k) {
  Slot &sl = s->slots[k];
  cudaStream_t st = sl.stream[r.tier];
  unsigned char *mem = s->d_arena + r.off;
  float *image = reinterpret_cast<float *>(mem);
  lrvol_step step = r.step;
  CU(cudaMemsetAsync(sl.d_scratch, 0, kSlotScratchBytes, st), "server: clear slot counters");
  CU(cudaEventRecord(sl.ev0, st), "server: record start");
  if (r.learned_auto) {
    float *feat = reinterpret_cast<float *>(mem + align256(r.image_bytes));
    float *mult = reinterpret_cast<float *>(mem + align256(r.image_bytes) + align256(r.vol->n_elem * 16 * 4));
    FeatureParams fp;
    int rc = prepare_features(r.vol, &r.cam, &r.tf, &step, &fp);
    if (rc) return rc;
    CU(launch_features(fp, feat, st), "server: features kernel");
    CU(launch_mlp_infer(feat, r.vol->n_elem, s->packed, s->ymin, s->ymax, mult,
                        reinterpret_cast<uint32_t *>(sl.d_scratch + 64), st),
       "server: network kernel");
    step.mult = mult;
  }
  RenderParams prm;
  int field = 0;
  int rc = prepare_render(r.vol, &r.cam, &r.tf, &step, image, &prm, &field);
  if (rc) return rc;
  if (prm.row_begin > 0 || prm.row_end < prm.height)  // rows outside the range read as transparent black
    CU(cudaMemsetAsync(image, 0, (size_t)r.image_bytes, st), "server: clear image");
  prm.counters = reinterpret_cast<unsigned long long *>(sl.d_scratch);
  prm.status = reinterpret_cast<uint32_t *>(sl.d_scratch + 64);
  if (prm.row_end > prm.row_begin)
    CU(launch_render(prm, r.vol->p[0], field, r.vol->storage, st), "server: render kernel");
  CU(cudaMemcpyAsync(sl.h_scratch, sl.d_scratch, kSlotScratchBytes, cudaMemcpyDeviceToHost, st),
     "server: read counters");
  if (r.host_out)
    CU(cudaMemcpyAsync(r.host_out, image, (size_t)r.image_bytes, cudaMemcpyDeviceToHost, st),
       "server: image to host");
  CU(cudaEventRecord(sl.ev1, st), "server: record end");
  return LRVOL_OK;
}

void finish(lrvol_server_s *s, Request &r, int32_t state, int32_t status) {
  r.state = state;
  r.status = status;
  r.t_done = now_s();
  if (state == LRVOL_REQ_DONE) ++s->done;
  else ++s->failed;
  s->finished.push_back(r.ticket);
  // the image stays in the arena only for a successful frame without host_out
  if (r.off >= 0 && (state != LRVOL_REQ_DONE || r.host_out)) {
    s->arena.release(r.off);
    r.off = -1;
  }
}

int retire(lrvol_server_s *s, int32_t *n_retired) {
  int32_t n = 0;
  for (size_t k = 0; k < s->slots.size(); ++k) {
    Slot &sl = s->slots[k];
    if (sl.ticket < 0) continue;
    cudaError_t e = cudaEventQuery(sl.ev1);
    if (e == cudaErrorNotReady) continue;
    Request &r = s->req[sl.ticket];
    sl.ticket = -1;
    --s->running;
    --s->running_tier[r.tier];
    ++n;
    if (e != cudaSuccess) {
      finish(s, r, LRVOL_REQ_FAILED, cuda_fail(e, "server: frame"));
      continue;
    }
    const unsigned long long *c = reinterpret_cast<const unsigned long long *>(sl.h_scratch);
    uint32_t st = 0;
    std::memcpy(&st, sl.h_scratch + 64, sizeof(st));
    r.samples = (int64_t)c[kCntSamples];
    r.lookups = (int64_t)c[kCntLookups];
    r.rays = (int64_t)c[kCntRays];
    cudaEventElapsedTime(&r.device_ms, sl.ev0, sl.ev1);
    cudaEventElapsedTime(&r.dev_start_ms, s->base, sl.ev0);
    cudaEventElapsedTime(&r.dev_end_ms, s->base, sl.ev1);
    if (st == kStatusBounds) finish(s, r, LRVOL_REQ_FAILED, fail(LRVOL_ERR_BOUNDS, "a kernel bounds check tripped"));
    else if (st == kStatusTimeout) finish(s, r, LRVOL_REQ_FAILED, fail(LRVOL_ERR_TIMEOUT, "a ray hit its sample cap"));
    else finish(s, r, LRVOL_REQ_DONE, LRVOL_OK);
  }
  if (n_retired) *n_retired = n;
  return LRVOL_OK;
}

// Admission.  Each tier's queue is served in arrival order.  With
// priorities on, tiers are tried from the smallest frames up, and the
// largest tier may hold at most slots - max(1, slots / 4) slots, so small
// and medium frames always find a slot; a request that does not fit (slot
// or memory) waits at the head of its tier while smaller tiers go ahead.
// With priorities off every request is in the last tier: plain FIFO.
void admit(lrvol_server_s *s) {
  const int nslots = (int)s->slots.size();
  const int reserve = s->priority_pixels > 0 ? (nslots / 4 > 1 ? nslots / 4 : 1) : 0;
  int cap_large = nslots - reserve > 1 ? nslots - reserve : 1;
  if (s->priority_pixels > 0 && s->large_cap > 0 && s->large_cap < cap_large) cap_large = s->large_cap;
  for (bool progress = true; progress;) {
    progress = false;
    for (int tier = 0; tier < kTiers; ++tier) {
      if (s->queue[tier].empty()) continue;
      if (tier == kTiers - 1 && s->running_tier[tier] >= cap_large) continue;
      int k = -1;
      for (int q = 0; q < nslots; ++q)
        if (s->slots[q].ticket < 0) {
          k = q;
          break;
        }
      if (k < 0) return;  // no slot for anyone
      Request &r = s->req[s->queue[tier].front()];
      const int64_t off = s->arena.alloc(r.bytes);
      if (off < 0) continue;  // this tier's head waits for memory
      s->queue[tier].pop_front();
      r.off = off;
      r.slot = k;
      r.t_admit = now_s();
      if (s->arena.in_use > s->high_water) s->high_water = s->arena.in_use;
      progress = true;
      int rc = launch_request(s, r, k);
      if (rc) {
        finish(s, r, LRVOL_REQ_FAILED, rc);
        break;
      }
      r.state = LRVOL_REQ_RUNNING;
      s->slots[k].ticket = r.ticket;
      ++s->running_tier[r.tier];
      if (++s->running > s->max_running) s->max_running = s->running;
      break;  // start again from the smallest tier
    }
  }
}

}  // namespace

extern "C" {

int lrvol_arena_create(int64_t bytes, int64_t align, lrvol_arena_t *out) {
  if (!out) return fail(LRVOL_ERR_ARG, "null pointer");
  *out = nullptr;
  lrvol_arena_s *a = new lrvol_arena_s();
  if (!init_arena(a, bytes, align)) {
    delete a;
    return fail(LRVOL_ERR_ARG, "arena: bytes >= 1 and a power-of-two alignment");
  }
  *out = a;
  return LRVOL_OK;
}

int64_t lrvol_arena_alloc(lrvol_arena_t a, int64_t bytes) { return a ? a->alloc(bytes) : -1; }

int lrvol_arena_free(lrvol_arena_t a, int64_t offset) {
  if (!a || !a->release(offset)) return fail(LRVOL_ERR_ARG, "arena: no block at this offset");
  return LRVOL_OK;
}

int64_t lrvol_arena_used(lrvol_arena_t a) { return a ? a->in_use : 0; }
int64_t lrvol_arena_largest_free(lrvol_arena_t a) { return a ? a->largest_free() : 0; }
void lrvol_arena_destroy(lrvol_arena_t a) { delete a; }

double lrvol_server_clock(void) { return now_s(); }

int lrvol_server_create(int32_t slots, int64_t arena_bytes, lrvol_server_t *out) {
  if (!out) return fail(LRVOL_ERR_ARG, "null pointer");
  *out = nullptr;
  if (slots < 1 || slots > 64) return fail(LRVOL_ERR_ARG, "slots must be 1..64");
  if (arena_bytes < ((int64_t)1 << 20)) return fail(LRVOL_ERR_ARG, "arena must be at least 1 MiB");
  lrvol_server_s *s = new lrvol_server_s();
  cudaGetDevice(&s->device);
  init_arena(&s->arena, arena_bytes, 256);
  s->slots.resize(slots);
  auto bail = [&](cudaError_t e, const char *what) {
    free_server(s);
    return cuda_fail(e, what);
  };
  cudaError_t e;
  int prio_low = 0, prio_high = 0;  // numerically lower is higher priority
  if ((e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high)) != cudaSuccess) return bail(e, "server: priorities");
  if ((e = cudaMalloc((void **)&s->d_arena, (size_t)arena_bytes)) != cudaSuccess) return bail(e, "server: arena");
  if ((e = cudaMalloc((void **)&s->d_scratch, (size_t)slots * kSlotScratchBytes)) != cudaSuccess)
    return bail(e, "server: slot scratch");
  if ((e = cudaMallocHost((void **)&s->h_scratch, (size_t)slots * kSlotScratchBytes)) != cudaSuccess)
    return bail(e, "server: pinned slot scratch");
  for (int k = 0; k < slots; ++k) {
    Slot &sl = s->slots[k];
    for (int t = 0; t < kTiers; ++t) {
      // tier 0 at the greatest priority, the last tier at the least, the middle between
      const int prio = prio_high + (prio_low - prio_high) * t / (kTiers - 1);
      if ((e = cudaStreamCreateWithPriority(&sl.stream[t], cudaStreamNonBlocking, prio)) != cudaSuccess)
        return bail(e, "server: streams");
    }
    if ((e = cudaEventCreate(&sl.ev0)) != cudaSuccess || (e = cudaEventCreate(&sl.ev1)) != cudaSuccess)
      return bail(e, "server: events");
    sl.d_scratch = s->d_scratch + (size_t)k * kSlotScratchBytes;
    sl.h_scratch = s->h_scratch + (size_t)k * kSlotScratchBytes;
  }
  if ((e = cudaEventCreate(&s->base)) != cudaSuccess) return bail(e, "server: base event");
  if ((e = cudaEventRecord(s->base, s->slots[0].stream[0])) != cudaSuccess) return bail(e, "server: base event");
  if ((e = cudaStreamSynchronize(s->slots[0].stream[0])) != cudaSuccess) return bail(e, "server: base event");
  *out = s;
  return LRVOL_OK;
}

int lrvol_server_set_step_model(lrvol_server_t s, const uint16_t *packed_dev, float ymin, float ymax) {
  if (!s || !packed_dev) return fail(LRVOL_ERR_ARG, "null pointer");
  if (reinterpret_cast<uintptr_t>(packed_dev) & 15) return fail(LRVOL_ERR_ARG, "packed weights must be 16-byte aligned");
  if (!(ymax >= 0.f && ymax <= 8.f)) return fail(LRVOL_ERR_ARG, "ymax must be in [0, 8]");
  if (!(ymin >= -8.f && ymin <= 0.f)) return fail(LRVOL_ERR_ARG, "ymin must be in [-8, 0]");
  s->packed = packed_dev;
  s->ymin = ymin;
  s->ymax = ymax;
  return LRVOL_OK;
}

int lrvol_server_set_priority_pixels(lrvol_server_t s, int64_t max_pixels) {
  if (!s || max_pixels < 0) return fail(LRVOL_ERR_ARG, "bad arguments");
  s->priority_pixels = max_pixels;
  return LRVOL_OK;
}

int lrvol_server_set_large_cap(lrvol_server_t s, int32_t max_in_flight) {
  if (!s || max_in_flight < 0) return fail(LRVOL_ERR_ARG, "bad arguments");
  s->large_cap = max_in_flight;
  return LRVOL_OK;
}

int lrvol_server_submit(lrvol_server_t s, lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf,
                        const lrvol_step *step, float *host_out, int64_t *ticket) {
  if (!s || !vol || !cam || !tf || !step || !ticket) return fail(LRVOL_ERR_ARG, "null pointer");
  Request r;
  r.vol = vol;
  r.cam = *cam;
  r.tf = *tf;
  r.step = *step;
  r.host_out = host_out;
  r.learned_auto = step->mode == LRVOL_STEP_LEARNED && step->mult == nullptr;
  const int64_t px = (int64_t)cam->width * cam->height;
  r.tier = px <= s->priority_pixels ? 0 : (px <= 4 * s->priority_pixels ? 1 : 2);
  if (r.learned_auto && !s->packed) return fail(LRVOL_ERR_STATE, "learned steps without multipliers need a step model");
  // the checks of lrvol_render, on placeholders for the memory the server provides
  lrvol_step chk = r.step;
  if (r.learned_auto) chk.mult = reinterpret_cast<const float *>(s->d_arena);
  RenderParams prm;
  int field = 0;
  int rc = prepare_render(vol, cam, tf, &chk, reinterpret_cast<float *>(s->d_arena), &prm, &field);
  if (rc) return rc;
  if (r.learned_auto) {
    FeatureParams fp;
    if ((rc = prepare_features(vol, cam, tf, &chk, &fp))) return rc;
  }
  r.image_bytes = (int64_t)cam->width * cam->height * 4 * (int64_t)sizeof(float);
  r.bytes = r.image_bytes;
  if (r.learned_auto) r.bytes = align256(r.image_bytes) + align256(vol->n_elem * 16 * 4) + align256(vol->n_elem * 4);
  if (s->arena.round(r.bytes) > s->arena.size) return fail(LRVOL_ERR_ARG, "request needs more memory than the arena");
  r.ticket = s->next_ticket++;
  r.t_submit = now_s();
  s->req[r.ticket] = r;
  s->queue[r.tier].push_back(r.ticket);
  ++s->submitted;
  *ticket = r.ticket;
  return LRVOL_OK;
}

int lrvol_server_progress(lrvol_server_t s, int32_t *n_retired) {
  if (!s) return fail(LRVOL_ERR_ARG, "null pointer");
  retire(s, n_retired);
  admit(s);
  return LRVOL_OK;
}

int lrvol_server_drain(lrvol_server_t s) {
  if (!s) return fail(LRVOL_ERR_ARG, "null pointer");
  for (;;) {
    retire(s, nullptr);
    admit(s);
    if (s->running == 0) {
      bool empty = true;
      for (int t = 0; t < kTiers; ++t) empty = empty && s->queue[t].empty();
      if (empty) return LRVOL_OK;
      return fail(LRVOL_ERR_OOM, "server: queued requests do not fit beside unreleased frames");
    }
    // wait for the oldest running frame
    int k = -1;
    int64_t oldest = INT64_MAX;
    for (size_t q = 0; q < s->slots.size(); ++q)
      if (s->slots[q].ticket >= 0 && s->slots[q].ticket < oldest) {
        oldest = s->slots[q].ticket;
        k = (int)q;
      }
    cudaEventSynchronize(s->slots[k].ev1);
  }
}

int lrvol_server_poll(lrvol_server_t s, int64_t *tickets, int32_t max_n, int32_t *n) {
  if (!s || !n || (max_n > 0 && !tickets)) return fail(LRVOL_ERR_ARG, "null pointer");
  int32_t k = 0;
  while (k < max_n && !s->finished.empty()) {
    tickets[k++] = s->finished.front();
    s->finished.pop_front();
  }
  *n = k;
  return LRVOL_OK;
}

int lrvol_server_info(lrvol_server_t s, int64_t ticket, lrvol_frame_info *info) {
  if (!s || !info) return fail(LRVOL_ERR_ARG, "null pointer");
  auto it = s->req.find(ticket);
  if (it == s->req.end()) return fail(LRVOL_ERR_ARG, "unknown ticket");
  const Request &r = it->second;
  std::memset(info, 0, sizeof(*info));
  info->state = r.state;
  info->status = r.status;
  info->rgba_dev = (r.state == LRVOL_REQ_DONE && r.off >= 0) ? reinterpret_cast<const float *>(s->d_arena + r.off)
                                                             : nullptr;
  info->t_submit = r.t_submit;
  info->t_admit = r.t_admit;
  info->t_done = r.t_done;
  info->device_ms = r.device_ms;
  info->dev_start_ms = r.dev_start_ms;
  info->dev_end_ms = r.dev_end_ms;
  info->samples = r.samples;
  info->lookups = r.lookups;
  info->rays_hit = r.rays;
  info->bytes = s->arena.round(r.bytes);
  return LRVOL_OK;
}

int lrvol_server_release(lrvol_server_t s, int64_t ticket) {
  if (!s) return fail(LRVOL_ERR_ARG, "null pointer");
  auto it = s->req.find(ticket);
  if (it == s->req.end()) return fail(LRVOL_ERR_ARG, "unknown ticket");
  Request &r = it->second;
  if (r.state == LRVOL_REQ_QUEUED || r.state == LRVOL_REQ_RUNNING)
    return fail(LRVOL_ERR_STATE, "request still queued or running");
  if (r.off >= 0) s->arena.release(r.off);
  s->req.erase(it);
  return LRVOL_OK;
}

int lrvol_server_get_stats(lrvol_server_t s, lrvol_server_stats *out) {
  if (!s || !out) return fail(LRVOL_ERR_ARG, "null pointer");
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  for (int t = 0; t < kTiers; ++t) out->queued += (int64_t)s->queue[t].size();
  out->running = s->running;
  out->done = s->done;
  out->failed = s->failed;
  out->arena_bytes = s->arena.size;
  out->arena_used = s->arena.in_use;
  out->arena_high_water = s->high_water;
  out->slots = (int32_t)s->slots.size();
  out->max_running = s->max_running;
  return LRVOL_OK;
}

void lrvol_server_destroy(lrvol_server_t s) {
  if (s) free_server(s);
}

}  // extern "C"
