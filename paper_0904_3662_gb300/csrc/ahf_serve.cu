// Serving front end: continuous batching of one-halo requests.
//
// The paper analyses a whole snapshot in one pass and has no serving layer;
// this one exists for callers that produce candidate haloes over time (an
// in-situ finder, an interactive catalogue service).  Each request is one
// halo with its candidates.  A worker thread packs the queued requests into
// batches and runs each batch through ahf_unbind_batch, forming and copying
// the next batch while the previous one computes (two batches in flight).
//
// Memory.  A request holds slots in two rings from submission until its
// batch has completed.  The device ring, sized from the caller's
// device-memory cap (particle state of every request in flight, its bound
// list, the result records and the context's workspace), is the admission
// rule: a request whose candidates do not fit in the device memory left is
// refused with AHF_ERR_FULL (the caller polls and retries).  The pinned host
// ring (at most 2^23 slots) stages the candidates at submission and takes
// the bound lists back; it refuses the same way when it is full.  A batch is
// a run of requests contiguous in both rings: one copy per array in, one
// copy of the bound lists out.  Slots return in submission order.
//
// Latency of a request = time from entering ahf_serve_submit to the moment
// its result became visible to ahf_serve_poll.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ahf_internal.h"

using namespace ahf;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int DEPTH = 2;                        // batches in flight
constexpr int64_t MAX_HOST_SLOTS = 1LL << 23;   // host staging ring (pinned memory)
constexpr int64_t MAX_DEV_SLOTS = 1LL << 31;    // device ring
constexpr int64_t MAX_BATCH_HALOS = 8192;
constexpr int64_t MAX_REQUEST = 131072;         // the on-chip classes' largest halo
constexpr size_t WS_RESERVE = 64ull << 20;      // allowance for the context's workspace

struct Req {
  uint64_t id = 0;
  int64_t start = 0, n = 0;  // device ring slots [start, start + max(n, 1))
  int64_t hstart = 0;        // host ring slots [hstart, hstart + max(n, 1))
  int64_t first = 0;         // caller's index of the first candidate
  double c[3] = {0.0, 0.0, 0.0};
  double radius = 0.0;
  Clock::time_point t_submit, t_done;
  bool done = false;
  int rc = AHF_OK;
  std::string err;
  ahf_result res{};
  std::vector<int64_t> bound;
};

// Slot ranges handed out and returned in FIFO order.
struct Ring {
  int64_t cap = 0, head = 0;
  std::deque<std::pair<int64_t, int64_t>> live;
  int64_t alloc(int64_t n) {
    if (n <= 0 || n > cap) return -1;
    int64_t start;
    if (live.empty()) {
      start = 0;
    } else {
      const int64_t tail = live.front().first;
      if (head > tail) {                      // used: [tail, head)
        if (head + n <= cap) start = head;
        else if (n <= tail) start = 0;        // wrap
        else return -1;
      } else {                                // wrapped: used [tail, cap) and [0, head)
        if (head + n <= tail) start = head;
        else return -1;
      }
    }
    live.emplace_back(start, start + n);
    head = start + n;
    return start;
  }
  void release_front() {
    live.pop_front();
    if (live.empty()) head = 0;
  }
  void undo_last() {                          // take back the range alloc just handed out
    live.pop_back();
    head = live.empty() ? 0 : live.back().second;
  }
};

struct Batch {
  std::vector<Req*> reqs;
  int64_t b0 = 0, b1 = 0;  // device ring range
  int64_t h0 = 0, h1 = 0;  // host ring range
  int slot = 0;
  int rc = AHF_OK;
  std::string err;
};

}  // namespace

struct ahf_serve {
  int device = 0;
  ahf_params prm{};
  int32_t coord_type = 0;
  double m0 = 0.0;        // > 0: uniform particle mass, requests carry no masses
  size_t es = 4;          // bytes per coordinate / velocity / mass element
  int n_arr = 6;          // arrays per candidate (7 with masses)
  int64_t S = 0;          // device ring slots
  int64_t SH = 0;         // host ring slots
  int64_t max_batch_slots = 0;
  ahf_ctx* ctx = nullptr;
  cudaStream_t ks = nullptr, cs = nullptr;  // compute / copy streams
  char* d_arena = nullptr;                  // n_arr arrays of S elements, then S int64 bound indices
  char* h_arena = nullptr;                  // pinned host copy of the same layout
  ahf_result* d_res = nullptr;              // DEPTH x MAX_BATCH_HALOS
  ahf_result* h_res = nullptr;
  cudaEvent_t ev_in[DEPTH] = {};
  cudaEvent_t ev_done[DEPTH] = {};
  std::vector<ahf_halo> hal[DEPTH];
  Batch batch[DEPTH];
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;
  std::atomic<int64_t> queued{0};
  std::unordered_map<uint64_t, Req*> reqs;
  Ring ring;              // device slots (the HBM cap)
  Ring hring;             // host staging slots
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // statistics since creation or the last reset
  std::vector<double> lat_us;
  int64_t submitted = 0, completed = 0, rejected = 0, batches = 0;
  Clock::time_point t_first, t_last;
  bool have_first = false;

  char* d_array(int a) const { return d_arena + (size_t)a * S * es; }
  char* h_array(int a) const { return h_arena + (size_t)a * SH * es; }
  int64_t* d_bound() const { return (int64_t*)(d_arena + (size_t)n_arr * S * es); }
  int64_t* h_bound() const { return (int64_t*)(h_arena + (size_t)n_arr * SH * es); }
};

namespace {

// Enqueue a batch: copy its ring slice in, unbind, copy results out.
void launch(ahf_serve* s, Batch* b) {
  const int k = b->slot;
  const int64_t n = b->b1 - b->b0;
  b->rc = AHF_OK;
  b->err.clear();
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < s->n_arr && e == cudaSuccess; ++a)
    e = cudaMemcpyAsync(s->d_array(a) + (size_t)b->b0 * s->es, s->h_array(a) + (size_t)b->h0 * s->es,
                        (size_t)n * s->es, cudaMemcpyHostToDevice, s->cs);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev_in[k], s->cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->ks, s->ev_in[k], 0);
  if (e != cudaSuccess) {
    b->rc = AHF_ERR_CUDA;
    b->err = std::string("serve input copy: ") + cudaGetErrorString(e);
  }
  if (b->rc == AHF_OK) {
    std::vector<ahf_halo>& H = s->hal[k];
    H.resize(b->reqs.size());
    for (size_t i = 0; i < b->reqs.size(); ++i) {
      const Req* r = b->reqs[i];
      H[i] = ahf_halo{r->c[0], r->c[1], r->c[2], r->radius, r->start, r->n};
    }
    ahf_particles P{};
    P.x = s->d_array(0);
    P.y = s->d_array(1);
    P.z = s->d_array(2);
    P.vx = s->d_array(3);
    P.vy = s->d_array(4);
    P.vz = s->d_array(5);
    P.m = s->n_arr == 7 ? s->d_array(6) : nullptr;
    P.m0 = s->m0;
    P.n = s->S;
    P.coord_type = s->coord_type;
    ahf_result* dres = s->d_res + (size_t)k * MAX_BATCH_HALOS;
    const int rc = ahf_unbind_batch(s->ctx, &P, H.data(), (int64_t)H.size(), nullptr, &s->prm, dres, s->d_bound(),
                                    nullptr, nullptr, s->ks);
    if (rc != AHF_OK) {
      b->rc = rc;
      b->err = ahf_last_error();
    } else {
      e = cudaMemcpyAsync(s->h_res + (size_t)k * MAX_BATCH_HALOS, dres, H.size() * sizeof(ahf_result),
                          cudaMemcpyDeviceToHost, s->ks);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_bound() + b->h0, s->d_bound() + b->b0, (size_t)n * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s->ks);
      if (e != cudaSuccess) {
        b->rc = AHF_ERR_CUDA;
        b->err = std::string("serve output copy: ") + cudaGetErrorString(e);
      }
    }
  }
  e = cudaEventRecord(s->ev_done[k], s->ks);
  if (e != cudaSuccess && b->rc == AHF_OK) {
    b->rc = AHF_ERR_CUDA;
    b->err = std::string("serve event: ") + cudaGetErrorString(e);
  }
}

// Move a completed batch's results into its requests and release its slots.
void finalize(ahf_serve* s, Batch* b, cudaError_t q) {
  if (q != cudaSuccess && b->rc == AHF_OK) {
    b->rc = AHF_ERR_CUDA;
    b->err = std::string("serve batch: ") + cudaGetErrorString(q);
  }
  const ahf_result* R = s->h_res + (size_t)b->slot * MAX_BATCH_HALOS;
  const int64_t* hb = s->h_bound();
  for (size_t i = 0; i < b->reqs.size(); ++i) {
    Req* r = b->reqs[i];
    r->rc = b->rc;
    if (b->rc != AHF_OK) {
      r->err = b->err;
      continue;
    }
    r->res = R[i];
    const int64_t nb = std::max<int64_t>(0, std::min<int64_t>(R[i].n_bound, r->n));
    r->bound.resize((size_t)nb);
    for (int64_t j = 0; j < nb; ++j) r->bound[(size_t)j] = hb[r->hstart + j] - r->start + r->first;
  }
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> g(s->mu);
  for (Req* r : b->reqs) {
    r->done = true;
    r->t_done = now;
    s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
    s->ring.release_front();
    s->hring.release_front();
  }
  s->completed += (int64_t)b->reqs.size();
  s->batches += 1;
  s->t_last = now;
}

void worker_main(ahf_serve* s) {
  cudaSetDevice(s->device);
  std::deque<Batch*> inflight;
  for (;;) {
    Batch* nb = nullptr;
    if ((int)inflight.size() < DEPTH && (inflight.empty() || s->queued.load(std::memory_order_acquire) > 0)) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (inflight.empty()) s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (inflight.empty() && s->queue.empty()) break;  // stopped and drained
      if (!s->queue.empty()) {
        int slot = 0;
        while (std::any_of(inflight.begin(), inflight.end(), [&](const Batch* x) { return x->slot == slot; }))
          ++slot;
        nb = &s->batch[slot];
        nb->slot = slot;
        nb->reqs.clear();
        nb->b0 = nb->b1 = s->queue.front()->start;
        nb->h0 = nb->h1 = s->queue.front()->hstart;
        while (!s->queue.empty() && (int64_t)nb->reqs.size() < MAX_BATCH_HALOS) {
          Req* r = s->queue.front();
          const int64_t len = std::max<int64_t>(r->n, 1);
          if (r->start != nb->b1 || r->hstart != nb->h1) break;   // a ring wrapped: next batch
          if (!nb->reqs.empty() && r->start + len - nb->b0 > s->max_batch_slots) break;
          nb->reqs.push_back(r);
          nb->b1 = r->start + len;
          nb->h1 = r->hstart + len;
          s->queue.pop_front();
        }
        s->queued.fetch_sub((int64_t)nb->reqs.size(), std::memory_order_release);
      }
    }
    if (nb) {
      launch(s, nb);
      inflight.push_back(nb);
      continue;
    }
    Batch* b = inflight.front();
    const cudaError_t q = cudaEventQuery(s->ev_done[b->slot]);
    if (q == cudaErrorNotReady) {
      std::this_thread::yield();
      continue;
    }
    finalize(s, b, q);
    inflight.pop_front();
  }
}

int check_params(const ahf_params* prm) {
  if (!prm) return set_last_error_fmt(AHF_ERR_INVALID, "params is NULL");
  if (prm->max_iter < 1) return set_last_error_fmt(AHF_ERR_INVALID, "max_iter < 1");
  if (prm->precision != AHF_PREC_MIXED && prm->precision != AHF_PREC_FP64)
    return set_last_error_fmt(AHF_ERR_INVALID, "unknown precision %d", prm->precision);
  if (prm->variant & ~(AHF_VAR_VBULK_INITIAL | AHF_VAR_RETRUNCATE | AHF_VAR_RISE_EDGE))
    return set_last_error_fmt(AHF_ERR_INVALID, "unknown variant bits %d", prm->variant);
  if (prm->reserved != 0) return set_last_error_fmt(AHF_ERR_INVALID, "params.reserved must be 0");
  return AHF_OK;
}

void release(ahf_serve* s) {
  for (auto& kv : s->reqs) delete kv.second;
  s->reqs.clear();
  for (int k = 0; k < DEPTH; ++k) {
    if (s->ev_in[k]) cudaEventDestroy(s->ev_in[k]);
    if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
  }
  if (s->ks) cudaStreamDestroy(s->ks);
  if (s->cs) cudaStreamDestroy(s->cs);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->d_res) cudaFree(s->d_res);
  if (s->h_arena) cudaFreeHost(s->h_arena);
  if (s->h_res) cudaFreeHost(s->h_res);
  if (s->ctx) ahf_destroy(s->ctx);
  delete s;
}

}  // namespace

extern "C" {

int ahf_serve_create(ahf_serve** out, int device, size_t hbm_cap_bytes, const ahf_params* prm,
                     int32_t coord_type, double m0) {
  if (!out) return set_last_error_fmt(AHF_ERR_INVALID, "serve handle is NULL");
  *out = nullptr;
  int rc = check_params(prm);
  if (rc != AHF_OK) return rc;
  if (coord_type != AHF_COORD_F64 && coord_type != AHF_COORD_F32_REL && coord_type != AHF_COORD_F32_BOX)
    return set_last_error_fmt(AHF_ERR_INVALID, "unknown coord_type %d", coord_type);
  if (!(m0 >= 0.0)) return set_last_error_fmt(AHF_ERR_INVALID, "m0 < 0");
  const size_t es = coord_type == AHF_COORD_F64 ? 8 : 4;
  const int n_arr = m0 > 0.0 ? 6 : 7;
  const size_t per_slot = (size_t)n_arr * es + sizeof(int64_t);
  const size_t fixed = WS_RESERVE + (size_t)DEPTH * MAX_BATCH_HALOS * sizeof(ahf_result);
  int64_t S = hbm_cap_bytes > fixed ? (int64_t)((hbm_cap_bytes - fixed) / per_slot) : 0;
  S = std::min(S, MAX_DEV_SLOTS) / 256 * 256;
  const int64_t SH = std::min(S, MAX_HOST_SLOTS);
  if (S < MAX_REQUEST)
    return set_last_error_fmt(AHF_ERR_INVALID, "hbm_cap_bytes %zu leaves %lld slots, below the %lld a request may need",
                              hbm_cap_bytes, (long long)S, (long long)MAX_REQUEST);
  ahf_serve* s = new (std::nothrow) ahf_serve();
  if (!s) return set_last_error_fmt(AHF_ERR_NOMEM, "serve allocation");
  s->device = device;
  s->prm = *prm;
  s->coord_type = coord_type;
  s->m0 = m0;
  s->es = es;
  s->n_arr = n_arr;
  s->S = S;
  s->SH = SH;
  s->max_batch_slots = SH / 2;
  s->ring.cap = S;
  s->hring.cap = SH;
  rc = ahf_create(&s->ctx, device);
  if (rc != AHF_OK) {
    release(s);
    return rc;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, (size_t)S * per_slot);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_res, (size_t)DEPTH * MAX_BATCH_HALOS * sizeof(ahf_result));
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_arena, (size_t)SH * per_slot);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_res, (size_t)DEPTH * MAX_BATCH_HALOS * sizeof(ahf_result));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->ks, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking);
  for (int k = 0; k < DEPTH && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&s->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_done[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    const int code = e == cudaErrorMemoryAllocation ? AHF_ERR_NOMEM : AHF_ERR_CUDA;
    set_last_error_fmt(code, "serve set-up (%lld slots): %s", (long long)S, cudaGetErrorString(e));
    release(s);
    return code;
  }
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    release(s);
    return set_last_error_fmt(AHF_ERR_NOMEM, "serve worker thread");
  }
  *out = s;
  return AHF_OK;
}

int ahf_serve_submit(ahf_serve* s, const ahf_particles* p, const ahf_halo* h, uint64_t* req_id) {
  const Clock::time_point t0 = Clock::now();
  if (!s || !p || !h || !req_id) return set_last_error_fmt(AHF_ERR_INVALID, "NULL argument");
  if (p->coord_type != s->coord_type)
    return set_last_error_fmt(AHF_ERR_INVALID, "coord_type %d, the serving instance takes %d", p->coord_type,
                              s->coord_type);
  if ((p->m == nullptr) != (s->n_arr == 6))
    return set_last_error_fmt(AHF_ERR_INVALID, s->n_arr == 6 ? "this instance takes no per-particle masses"
                                                             : "this instance needs per-particle masses");
  if (s->n_arr == 6 && p->m0 != s->m0)
    return set_last_error_fmt(AHF_ERR_INVALID, "m0 %g differs from the instance's %g", p->m0, s->m0);
  if (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz) return set_last_error_fmt(AHF_ERR_INVALID, "NULL array");
  if (p->u_th) return set_last_error_fmt(AHF_ERR_INVALID, "serving takes no gas thermal energies (u_th)");
  if (h->offset < 0 || h->count < 0 || h->offset + h->count > p->n)
    return set_last_error_fmt(AHF_ERR_INVALID, "halo slots [%lld, %lld) outside the %lld particles",
                              (long long)h->offset, (long long)(h->offset + h->count), (long long)p->n);
  if (h->count > MAX_REQUEST)
    return set_last_error_fmt(AHF_ERR_INVALID, "%lld candidates above the serving limit %lld (use ahf_unbind_batch)",
                              (long long)h->count, (long long)MAX_REQUEST);
  if (!(h->radius >= 0.0)) return set_last_error_fmt(AHF_ERR_INVALID, "radius < 0");
  Req* r = new (std::nothrow) Req();
  if (!r) return set_last_error_fmt(AHF_ERR_NOMEM, "request record");
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) {
    delete r;
    return set_last_error_fmt(AHF_ERR_INVALID, "serving instance is shutting down");
  }
  const int64_t len = std::max<int64_t>(h->count, 1);
  const int64_t start = s->ring.alloc(len);
  if (start < 0) {
    delete r;
    s->rejected += 1;
    return set_last_error_fmt(AHF_ERR_FULL, "no room for %lld candidates in the device memory cap (%lld slots); "
                              "poll and retry", (long long)h->count, (long long)s->S);
  }
  const int64_t hstart = s->hring.alloc(len);
  if (hstart < 0) {
    s->ring.undo_last();
    delete r;
    s->rejected += 1;
    return set_last_error_fmt(AHF_ERR_FULL, "no room for %lld candidates in the %lld-slot host staging ring; "
                              "poll and retry", (long long)h->count, (long long)s->SH);
  }
  const void* src[7] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->m};
  for (int a = 0; a < s->n_arr; ++a)
    std::memcpy(s->h_array(a) + (size_t)hstart * s->es, (const char*)src[a] + (size_t)h->offset * s->es,
                (size_t)h->count * s->es);
  r->id = s->next_id++;
  r->start = start;
  r->hstart = hstart;
  r->n = h->count;
  r->first = h->offset;
  r->c[0] = h->cx;
  r->c[1] = h->cy;
  r->c[2] = h->cz;
  r->radius = h->radius;
  r->t_submit = t0;
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  s->queued.fetch_add(1, std::memory_order_release);
  s->submitted += 1;
  if (!s->have_first) {
    s->have_first = true;
    s->t_first = t0;
  }
  *req_id = r->id;
  s->cv.notify_one();
  return AHF_OK;
}

int ahf_serve_poll(ahf_serve* s, uint64_t req_id, ahf_result* out_host, int64_t* bound_idx_host, int64_t cap) {
  if (!s) return set_last_error_fmt(AHF_ERR_INVALID, "serve handle is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return set_last_error_fmt(AHF_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
  Req* r = it->second;
  if (!r->done) return AHF_PENDING;
  if (r->rc != AHF_OK) {
    const int rc = r->rc;
    set_last_error_fmt(rc, "request %llu: %s", (unsigned long long)req_id, r->err.c_str());
    s->reqs.erase(it);
    delete r;
    return rc;
  }
  if (out_host) *out_host = r->res;
  const int64_t nb = (int64_t)r->bound.size();
  if (bound_idx_host) {
    if (cap < nb)
      return set_last_error_fmt(AHF_ERR_INVALID, "bound list of %lld entries does not fit cap %lld", (long long)nb,
                                (long long)cap);
    if (nb) std::memcpy(bound_idx_host, r->bound.data(), (size_t)nb * sizeof(int64_t));
  }
  s->reqs.erase(it);
  delete r;
  return AHF_OK;
}

int ahf_serve_stats(ahf_serve* s, double* p50_us, double* p99_us, double* throughput) {
  if (!s) return set_last_error_fmt(AHF_ERR_INVALID, "serve handle is NULL");
  std::vector<double> lat;
  double thr = 0.0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    lat = s->lat_us;
    if (s->completed > 0 && s->have_first) {
      const double sec = std::chrono::duration<double>(s->t_last - s->t_first).count();
      if (sec > 0.0) thr = (double)s->completed / sec;
    }
  }
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    size_t k = (size_t)std::ceil(q * (double)lat.size());
    k = std::min(std::max<size_t>(k, 1), lat.size()) - 1;
    std::nth_element(lat.begin(), lat.begin() + (long)k, lat.end());
    return lat[k];
  };
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  if (throughput) *throughput = thr;
  return AHF_OK;
}

int ahf_serve_counters(ahf_serve* s, int64_t* submitted, int64_t* completed, int64_t* rejected, int64_t* batches) {
  if (!s) return set_last_error_fmt(AHF_ERR_INVALID, "serve handle is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  if (submitted) *submitted = s->submitted;
  if (completed) *completed = s->completed;
  if (rejected) *rejected = s->rejected;
  if (batches) *batches = s->batches;
  return AHF_OK;
}

int ahf_serve_reset_stats(ahf_serve* s) {
  if (!s) return set_last_error_fmt(AHF_ERR_INVALID, "serve handle is NULL");
  std::lock_guard<std::mutex> g(s->mu);
  s->lat_us.clear();
  s->submitted = s->completed = s->rejected = s->batches = 0;
  s->have_first = false;
  return AHF_OK;
}

int ahf_serve_destroy(ahf_serve* s) {
  if (!s) return AHF_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  release(s);
  return AHF_OK;
}

}  // extern "C"
