// Host side of libahfgpu: the C ABI, argument validation, the size-class
// scheduler and the context's device workspace.
//
// Scheduling.  Haloes are independent units (the paper's parallel version
// relies on the same fact: no communication during the analysis, Sect. 2.2).
// Each halo goes to a size class by its candidate count: three on-chip
// variants (one CTA per halo, everything in shared memory) and, above the
// largest on-chip capacity, the multi-CTA class that streams its particles
// through HBM.  Within a class the haloes are processed largest first by
// persistent CTAs pulling from a device counter (longest-processing-time
// order), so the biggest halo starts first and the tail is short.
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "ahf_internal.h"

using namespace ahf;

#ifndef AHF_BUILD_ID
#define AHF_BUILD_ID "unknown"
#endif

namespace {

thread_local std::string g_last_error;
thread_local const char* g_last_ptr = "";

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  g_last_ptr = g_last_error.c_str();
  return code;
}

#define AHF_CUDA(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(AHF_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                         \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// A bump allocator over the context's device workspace, rebuilt per call.
struct Bump {
  char* base = nullptr;
  size_t used = 0;
  size_t cap = 0;
  template <typename T>
  T* take(size_t count) {
    used = align_up(used, 256);
    T* p = reinterpret_cast<T*>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

}  // namespace

void ahf::set_last_error_static(const char* msg) { g_last_ptr = msg; }

void ahf::profile_bin_tables(int n, double f, double* t) {
  for (int b = 0; b < n; ++b) t[b] = std::pow(f, 1.0 - (double)b / (double)n);
  for (int b = 0; b < n; ++b) {
    const double f0 = t[b], f1 = b + 1 < n ? t[b + 1] : 1.0;
    t[n + b] = 1.0 / (4.0 * M_PI / 3.0 * (f1 * f1 * f1 - f0 * f0 * f0));
    t[2 * n + b] = 1.0 / f1;
  }
}

int ahf::set_last_error_fmt(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  g_last_ptr = g_last_error.c_str();
  return code;
}

namespace {

// Shared-memory variants in size order: 0 = one warp per halo, 1-3 = one CTA
// of 128 / 256 / 512 threads, 4-6 = clusters of 4 / 8 / 16 CTAs.  Phases
// 0..NV-1 time them; then the multi-CTA class's three phases and the profile.
constexpr int NV = 8;
constexpr int PH_GRID_SORT = NV, PH_GRID_ITER = NV + 1, PH_GRID_FINISH = NV + 2, PH_PROFILE = NV + 3;
static_assert(PH_PROFILE + 1 == AHF_N_PHASES, "phase table");

int variant_capacity(int v) { return v == 0 ? warp_capacity() : onchip_capacity(v - 1); }

// Resident CTAs (whole clusters) of a variant on this device; 0 if it cannot run.
int variant_max_grid(int v, int device) { return v == 0 ? warp_max_grid(device) : onchip_max_grid(v - 1, device); }

// CTAs a launch of n haloes needs (before the residency cap).
long long variant_grid_for(int v, long long n) {
  if (v == 0) return (n + warp_halos_per_cta() - 1) / warp_halos_per_cta();
  return n * onchip_cluster_size(v - 1);
}

cudaError_t launch_variant(const OnchipLaunch& L, int v, int grid, cudaStream_t s) {
  return v == 0 ? launch_warp(L, grid, s) : launch_onchip(L, v - 1, grid, s);
}

}  // namespace

struct ahf_ctx {
  int device = 0;
  int sms = 0;
  char* ws = nullptr;            // device workspace
  size_t ws_bytes = 0;
  int* err_dev = nullptr;        // device error word
  int* err_host = nullptr;       // pinned mirror
  cudaEvent_t last = nullptr;    // end of the previous call's device work
  bool last_valid = false;
  int64_t onchip_max = 16 * 8192;    // largest candidate count of the shared-memory classes
  int64_t wait_limit = 1 << 22;      // polls of a tensor copy's barrier before a timeout
  int64_t class_cut[NV] = {-1, -1, -1, -1, -1, -1, -1, -1};  // largest count per on-chip variant (-1: capacity)
  int pass_chunk = 8;                // multi-CTA passes per read of the active count
  int64_t ws_cap = 0;                // largest workspace the context may hold (0: no cap)
  char tuning[512] = {};             // tuning file applied at creation ("" = none)
  std::mutex mu;
  // pinned staging for host descriptors: a ring of slots, each released by
  // an event after the copies that read it, so a call never waits for the
  // previous call's kernels just to reuse staging memory
  static constexpr int NPIN = 4;
  void* pin[NPIN] = {};
  size_t pin_bytes[NPIN] = {};
  cudaEvent_t pin_ev[NPIN] = {};
  bool pin_ev_valid[NPIN] = {};
  int pin_next = 0;
  int pin_cur = -1;
  int* flag_host = nullptr;      // pinned readback of small device words
  char* stage = nullptr;         // device staging of the host-memory entry point
  size_t stage_bytes = 0;
  // per-call statistics and optional phase timing
  bool timing = false;
  int host_direct = 2;               // host entry: 0 staged, 1 in place, 2 inputs in place + pushed outputs
  bool graphs = false;               // on-chip launch sequence as a replayed CUDA graph
  void* hier = nullptr;              // hierarchy scratch (owners, compacted member lists)
  size_t hier_bytes = 0;
  void* aux = nullptr;               // second-pass member lists (AHF_VAR_RETRUNCATE)
  size_t aux_bytes = 0;
  bool trace = false;                // per-halo timestamps from the on-chip kernels
  bool serial = false;               // on-chip classes one after another on the caller's stream
  bool promote = true;               // small batches take larger classes (lower latency)
  long long* trace_dev = nullptr;    // [n][AHF_TRACE_FIELDS] of the last traced call
  int64_t trace_cap = 0;             // haloes trace_dev holds
  int64_t trace_n = -1;              // haloes of the last traced call (-1: none)
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture = nullptr;    // stream the graph is captured on
  std::vector<unsigned char> graph_key;   // launch parameters the graph was captured with
  ahf_stats stats{};
  bool phase_used[AHF_N_PHASES] = {};
  cudaEvent_t ev0[AHF_N_PHASES] = {}, ev1[AHF_N_PHASES] = {};
  cudaStream_t side[NV] = {};    // one stream per shared-memory variant
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[NV] = {};
  int variant_grid[NV] = {-1, -1, -1, -1, -1, -1, -1, -1};   // resident CTAs per variant (-1: not queried)
  int iter_grid[2] = {-1, -1};       // CTAs of the multi-CTA pass (mixed, FP64; -1: not queried)
  int tma_grid = -1;                 // CTAs of the pass with tensor copies (-1: not queried)
  std::vector<HaloDev> plan_hd;      // host descriptor buffer reused by the calls' plans
};

namespace {

// Take the next staging slot (waiting only for that slot's own copies) with
// at least `bytes` of pinned memory; release with pin_release after the
// copies are enqueued.
int pin_acquire(ahf_ctx* c, size_t bytes, char** out) {
  const int k = c->pin_next;
  c->pin_next = (k + 1) % ahf_ctx::NPIN;
  if (c->pin_ev_valid[k]) AHF_CUDA(cudaEventSynchronize(c->pin_ev[k]));
  if (bytes > c->pin_bytes[k]) {
    if (c->pin[k]) cudaFreeHost(c->pin[k]);
    c->pin[k] = nullptr;
    c->pin_bytes[k] = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20);
    if (cudaMallocHost(&c->pin[k], want) != cudaSuccess) return fail(AHF_ERR_NOMEM, "pinned staging of %zu bytes", want);
    c->pin_bytes[k] = want;
  }
  c->pin_cur = k;
  *out = (char*)c->pin[k];
  return AHF_OK;
}

int pin_release(ahf_ctx* c, cudaStream_t s) {
  const int k = c->pin_cur;
  if (k < 0) return AHF_OK;
  AHF_CUDA(cudaEventRecord(c->pin_ev[k], s));
  c->pin_ev_valid[k] = true;
  c->pin_cur = -1;
  return AHF_OK;
}

int ensure_workspace(ahf_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return AHF_OK;
  if (c->ws_cap > 0 && bytes > (size_t)c->ws_cap)
    return fail(AHF_ERR_NOMEM, "the call needs %zu bytes of workspace, above the cap of %lld", bytes,
                (long long)c->ws_cap);
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  size_t want = std::max(align_up(bytes + bytes / 8, 1 << 20), (size_t)1 << 22);
  if (c->ws_cap > 0) want = std::max(bytes, std::min(want, (size_t)c->ws_cap));
  if (cudaMalloc(&c->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(AHF_ERR_NOMEM, "device workspace of %zu bytes", want);
  }
  c->ws_bytes = want;
  return AHF_OK;
}

void reset_stats(ahf_ctx* c) {
  c->stats = ahf_stats{};
  for (int k = 0; k < AHF_N_PHASES; ++k) {
    c->stats.phase_ms[k] = -1.0;
    c->phase_used[k] = false;
  }
}

int phase_begin(ahf_ctx* c, int ph, cudaStream_t s, long long halos, long long cands) {
  c->phase_used[ph] = true;
  c->stats.phase_halos[ph] += halos;
  c->stats.phase_candidates[ph] += cands;
  if (c->timing) AHF_CUDA(cudaEventRecord(c->ev0[ph], s));
  return AHF_OK;
}

int phase_end(ahf_ctx* c, int ph, cudaStream_t s) {
  if (c->timing) AHF_CUDA(cudaEventRecord(c->ev1[ph], s));
  return AHF_OK;
}

}  // namespace

namespace {

// 2^e as a double, e in [-1022, 1023]: x * pow2(e) is ldexp(x, e), the one
// rounding of the exact product (scaling by a power of two)
inline double pow2(int e) {
  const uint64_t b = (uint64_t)(e + 1023) << 52;
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
}

// llround for |v| < 2^63: nearest integer, halves away from zero (v minus
// its truncation is exact)
inline long long round_away(double v) {
  long long i = (long long)v;
  const double r = v - (double)i;
  if (r >= 0.5) ++i;
  else if (r <= -0.5) --i;
  return i;
}

}  // namespace

void ahf::fill_halo_dev(const ahf_halo& H, int coord_type, double box, int index, HaloDev& d) {
  d.c[0] = H.cx; d.c[1] = H.cy; d.c[2] = H.cz;
  // fixed-point frame of this halo alone (so a halo's result does not depend
  // on the rest of the batch): its centre, every member and the box stay
  // below 2^(60-frac)
  const double cm = std::max(std::fabs(H.cx), std::max(std::fabs(H.cy), std::fabs(H.cz)));
  double span = std::max(cm + std::fabs(H.radius), box);
  if (coord_type == AHF_COORD_F32_REL) span = std::max(span, 1.0);
  // e: the smallest integer with 2^e > span + 1 (span + 1 >= 1: from the
  // biased exponent while finite)
  const double s1 = span + 1.0;
  int e = 0;
  if (std::isfinite(s1)) {
    uint64_t b;
    std::memcpy(&b, &s1, sizeof b);
    e = (int)((b >> 52) & 0x7ff) - 1022;
  } else {
    std::frexp(s1, &e);
  }
  e = std::min(e, 1100);
  const int frac = std::max(-200, std::min(200, 60 - e));
  d.frac = frac;
  bool exact = coord_type != AHF_COORD_F64 && box == 0.0;
  for (int a = 0; a < 3; ++a) {
    d.cf[a] = (float)d.c[a];
    exact = exact && (double)d.cf[a] == d.c[a];
  }
  d.fast = exact ? 1 : 0;
  // the fixed-point frame (used only off the fast path); every value scaled
  // here is below 2^60 in magnitude
  const double sc = pow2(frac);
  d.boxfix = box > 0.0 ? round_away(box * sc) : 0;
  for (int a = 0; a < 3; ++a) d.cfix[a] = exact ? 0 : round_away(d.c[a] * sc);
  const double R = H.radius;
  d.R2 = R * R;
  d.R2lo = (float)(d.R2 * (1.0 - 4e-6));
  d.R2hi = (float)(d.R2 * (1.0 + 4e-6));
  d.offset = H.offset;
  d.count = H.count;
  d.gbase = 0;
  d.index = index;
}

namespace {

struct Plan {
  std::vector<HaloDev> hd;     // reordered: class 0, 1, 2 (on-chip), then grid class
  int n_class[NV + 1] = {};     // 0..NV-1 shared-memory variants, NV multi-CTA
  long long grid_flat = 0;
  long long onchip_flat = 0;     // candidates of the on-chip classes (their records)
  FrameDev frame;
  ahf_ctx* owner = nullptr;      // whose descriptor buffer hd holds
  Plan() = default;
  Plan(const Plan&) = delete;
  Plan& operator=(const Plan&) = delete;
  // the descriptor buffer goes back to the context for the next call (a
  // fresh 120-byte-per-halo array each call cost its page faults and zeroing)
  ~Plan() {
    if (owner && owner->plan_hd.capacity() < hd.capacity()) owner->plan_hd.swap(hd);
  }
};

int validate(const ahf_particles* p, const ahf_halo* halos, int64_t n_halos, const ahf_params* prm,
             const ahf_result* out, const int64_t* bound_idx) {
  if (!p || !prm) return fail(AHF_ERR_INVALID, "particles and params must not be NULL");
  if (n_halos < 0) return fail(AHF_ERR_INVALID, "n_halos < 0");
  if (n_halos > 0 && (!halos || !out || !bound_idx))
    return fail(AHF_ERR_INVALID, "halos, out and bound_idx must not be NULL");
  if (n_halos >= ((int64_t)1 << 27)) return fail(AHF_ERR_INVALID, "n_halos above 2^27-1");
  if (p->n < 0) return fail(AHF_ERR_INVALID, "particle count < 0");
  if (p->n > 0 && (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz))
    return fail(AHF_ERR_INVALID, "coordinate or velocity array is NULL");
  if (p->coord_type != AHF_COORD_F64 && p->coord_type != AHF_COORD_F32_REL && p->coord_type != AHF_COORD_F32_BOX)
    return fail(AHF_ERR_INVALID, "unknown coord_type %d", p->coord_type);
  if (p->reserved != 0) return fail(AHF_ERR_INVALID, "reserved field must be 0");
  if (!p->m && !(p->m0 >= 0.0 && std::isfinite(p->m0))) return fail(AHF_ERR_INVALID, "m0 must be finite and >= 0");
  if (prm->max_iter < 1) return fail(AHF_ERR_INVALID, "max_iter must be >= 1");
  if (prm->precision != AHF_PREC_MIXED && prm->precision != AHF_PREC_FP64)
    return fail(AHF_ERR_INVALID, "unknown precision mode %d", prm->precision);
  if (prm->variant & ~(AHF_VAR_VBULK_INITIAL | AHF_VAR_RETRUNCATE | AHF_VAR_RISE_EDGE))
    return fail(AHF_ERR_INVALID, "unknown variant bits %d", prm->variant);
  if (prm->reserved != 0) return fail(AHF_ERR_INVALID, "params.reserved must be 0");
  if (!(prm->G > 0.0) || !std::isfinite(prm->G)) return fail(AHF_ERR_INVALID, "G must be > 0");
  if (!std::isfinite(prm->H)) return fail(AHF_ERR_INVALID, "H must be finite");
  if (!(prm->delta_rho > 0.0) || !std::isfinite(prm->delta_rho)) return fail(AHF_ERR_INVALID, "delta_rho must be > 0");
  if (!(prm->r_soft >= 0.0) || !std::isfinite(prm->r_soft)) return fail(AHF_ERR_INVALID, "r_soft must be >= 0");
  if (!(prm->box >= 0.0) || !std::isfinite(prm->box)) return fail(AHF_ERR_INVALID, "box must be >= 0");
  if (!(prm->band >= 0.0) || !(prm->band < 1.0)) return fail(AHF_ERR_INVALID, "band must be in [0, 1)");
  return AHF_OK;
}

// Check slots: in range of the slot space and not shared between haloes.
int validate_slots(const ahf_halo* halos, int64_t n_halos, int64_t n_slots, bool have_members) {
  std::vector<std::pair<int64_t, int64_t>> iv;
  iv.reserve((size_t)n_halos);
  for (int64_t h = 0; h < n_halos; ++h) {
    const ahf_halo& H = halos[h];
    if (H.count < 0 || H.offset < 0) return fail(AHF_ERR_INVALID, "halo %lld: negative offset or count", (long long)h);
    if (H.count > (int64_t)0x7fffffff) return fail(AHF_ERR_INVALID, "halo %lld: count above 2^31-1", (long long)h);
    if (!have_members && H.offset + H.count > n_slots)
      return fail(AHF_ERR_INVALID, "halo %lld: slots [%lld, %lld) beyond %lld particles", (long long)h,
                  (long long)H.offset, (long long)(H.offset + H.count), (long long)n_slots);
    if (!(std::isfinite(H.cx) && std::isfinite(H.cy) && std::isfinite(H.cz)))
      return fail(AHF_ERR_INVALID, "halo %lld: centre not finite", (long long)h);
    if (!std::isfinite(H.radius)) return fail(AHF_ERR_INVALID, "halo %lld: radius must be finite", (long long)h);
    if (H.count > 0) iv.emplace_back(H.offset, H.offset + H.count);
  }
  // slots usually come in increasing order: sort only when they do not
  if (!std::is_sorted(iv.begin(), iv.end())) std::sort(iv.begin(), iv.end());
  for (size_t i = 1; i < iv.size(); ++i)
    if (iv[i].first < iv[i - 1].second) return fail(AHF_ERR_INVALID, "haloes share candidate slots");
  return AHF_OK;
}

// Ascending order of 64-bit keys whose low `low_bits` bits hold distinct
// positions already in ascending order (h = 0, 1, ...): a stable LSD radix
// sort on the higher bytes where the keys differ (the positions keep the
// order of equal higher parts), 256 counters per pass.  The keys are taken
// as four consecutive quarters, each with its own counters (the quarter's
// runs of every digit placed in quarter order, so the sort stays stable):
// the four counter updates of a step are independent, where one set of
// counters made every key wait for the previous key's update of the same
// digit.
void sort_plan_keys(std::vector<uint64_t>& key, int low_bits) {
  const size_t n = key.size();
  if (n < 2) return;
  uint64_t orb = 0, andb = ~0ull;
  for (uint64_t k : key) { orb |= k; andb &= k; }
  const uint64_t diff = orb ^ andb;
  std::vector<uint64_t> tmp(n);
  constexpr int Q = 4;
  const size_t q = n / Q;                // keys [Q q, n) follow the last quarter's
  for (int b = low_bits / 8; b < 8; ++b) {
    if (((diff >> (8 * b)) & 0xffull) == 0) continue;
    const int sh = 8 * b;
    uint32_t cnt[Q][256] = {};
    const uint64_t* k = key.data();
    for (size_t i = 0; i < q; ++i)
      for (int s = 0; s < Q; ++s) ++cnt[s][(k[s * q + i] >> sh) & 0xffu];
    for (size_t j = Q * q; j < n; ++j) ++cnt[Q - 1][(k[j] >> sh) & 0xffu];
    uint32_t run = 0;
    for (int d = 0; d < 256; ++d)
      for (int s = 0; s < Q; ++s) {
        const uint32_t c = cnt[s][d];
        cnt[s][d] = run;
        run += c;
      }
    uint64_t* t = tmp.data();
    for (size_t i = 0; i < q; ++i)
      for (int s = 0; s < Q; ++s) {
        const uint64_t x = k[s * q + i];
        t[cnt[s][(x >> sh) & 0xffu]++] = x;
      }
    for (size_t j = Q * q; j < n; ++j) t[cnt[Q - 1][(k[j] >> sh) & 0xffu]++] = k[j];
    key.swap(tmp);
  }
}

int make_plan(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos, const ahf_params* prm,
              Plan& P) {
  P.frame.box = prm->box;
  // the smallest shared-memory variant that holds the halo and can run on
  // this device, else the multi-CTA class
  int caps[NV];
  for (int v = 0; v < NV; ++v) {
    if (c->variant_grid[v] < 0) c->variant_grid[v] = variant_max_grid(v, c->device);
    caps[v] = c->variant_grid[v] > 0 ? (int)std::min<int64_t>(variant_capacity(v), c->onchip_max) : 0;
    if (c->class_cut[v] >= 0) caps[v] = (int)std::min<int64_t>(caps[v], c->class_cut[v]);
  }
  std::vector<int> cls((size_t)n_halos);
  for (int64_t h = 0; h < n_halos; ++h) {
    const int64_t n = halos[h].count;
    int k = NV;
    // the all-FP64 mode and gas (thermal energy per particle) run in the
    // multi-CTA class only
    if (prm->precision == AHF_PREC_MIXED && !p->u_th)
      for (int v = 0; v < NV; ++v)
        if (caps[v] > 0 && n <= caps[v]) { k = v; break; }
    cls[h] = k;
  }
  // latency: a batch that leaves SMs idle moves its haloes to larger classes
  // (more threads per halo; every class gives the same bits), at most two
  // classes up and to the 8-CTA cluster (the 16-CTA one for haloes that
  // start in a 4-CTA cluster or larger), while the whole batch still runs at
  // once
  if (c->promote) {
    double inflight[NV];
    for (int v = 0; v < NV; ++v)
      inflight[v] = v == 0 ? (double)c->variant_grid[0] * warp_halos_per_cta()
                           : (double)c->variant_grid[v] / onchip_cluster_size(v - 1);
    const std::vector<int> base = cls;
    for (int round = 0; round < 2; ++round) {
      std::vector<int> next = cls;
      double load = 0.0;
      bool moved = false;
      for (int64_t h = 0; h < n_halos; ++h) {
        const int k = cls[(size_t)h];
        if (k >= NV) continue;
        const int top = base[(size_t)h] >= 5 ? NV - 1 : 6;
        if (k + 1 <= top && caps[k + 1] > 0 && inflight[k + 1] >= 1.0) {
          next[(size_t)h] = k + 1;
          moved = true;
        }
        load += 1.0 / inflight[next[(size_t)h]];
      }
      if (!moved || load > 1.0) break;
      cls.swap(next);
    }
  }
  for (int64_t h = 0; h < n_halos; ++h) P.n_class[cls[(size_t)h]]++;
  // order: by class, largest first within a class (ties by input position),
  // as one sort of packed keys (class | ~count | position)
  std::vector<uint64_t> key((size_t)n_halos);
  for (int64_t h = 0; h < n_halos; ++h) {
    const uint64_t cnt = (uint64_t)std::min<int64_t>(halos[h].count, 0xffffffffll);
    key[(size_t)h] = ((uint64_t)cls[h] << 60) | ((0xffffffffull - cnt) << 27) | (uint64_t)h;
  }
  sort_plan_keys(key, 27);
  std::vector<int> order((size_t)n_halos);
  for (int64_t k = 0; k < n_halos; ++k) order[(size_t)k] = (int)(key[(size_t)k] & ((1ull << 27) - 1));
  P.owner = c;
  P.hd.swap(c->plan_hd);                 // sized by an earlier call: no zeroing
  P.hd.resize((size_t)n_halos);
  long long gbase = 0, rbase = 0;
  for (int64_t k = 0; k < n_halos; ++k) {
    const int h = order[k];
    const ahf_halo& H = halos[h];
    HaloDev& d = P.hd[k];
    fill_halo_dev(H, p->coord_type, prm->box, h, d);
    // multi-CTA haloes start on 8-element rows (the passes' tensor copies)
    if (cls[h] == NV) { d.gbase = gbase; gbase = (gbase + H.count + 7) & ~7ll; }
    else { d.gbase = rbase; rbase += H.count; }
  }
  P.grid_flat = gbase;
  P.onchip_flat = rbase;
  return AHF_OK;
}

// (the device structs are zeroed first: their bytes, padding included, are
// part of the graph key)
ParamsDev to_dev(const ahf_params* prm) {
  ParamsDev d;
  std::memset(&d, 0, sizeof d);
  d.G = prm->G; d.H = prm->H; d.delta_rho = prm->delta_rho; d.r_soft = prm->r_soft; d.band = prm->band;
  d.Gf = (float)prm->G; d.Hf = (float)prm->H; d.r_soft_f = (float)prm->r_soft; d.band_f = (float)prm->band;
  d.crit = prm->delta_rho * (4.0 * M_PI / 3.0);
  d.crit_f = (float)d.crit;
  d.inv_crit = 1.0 / d.crit;
  d.max_iter = prm->max_iter;
  d.precision = prm->precision;
  d.vbulk_initial = (prm->variant & AHF_VAR_VBULK_INITIAL) ? 1 : 0;
  d.rise_edge = (prm->variant & AHF_VAR_RISE_EDGE) ? 1 : 0;
  return d;
}

ParticlesDev to_dev(const ahf_particles* p) {
  ParticlesDev d;
  std::memset(&d, 0, sizeof d);
  d.x = p->x; d.y = p->y; d.z = p->z; d.vx = p->vx; d.vy = p->vy; d.vz = p->vz; d.m = p->m;
  d.u_th = p->u_th;
  d.m0 = p->m0; d.m0f = (float)p->m0; d.coord_type = p->coord_type; d.n = p->n;
  return d;
}

int begin_call(ahf_ctx* c, cudaStream_t s) {
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaStreamWaitEvent(s, c->last, 0));
  return AHF_OK;
}

int end_call(ahf_ctx* c, cudaStream_t s) {
  AHF_CUDA(cudaEventRecord(c->last, s));
  c->last_valid = true;
  return AHF_OK;
}

// Sizes of the multi-CTA class's workspace for one call.
struct GridSizes {
  size_t nf = 0;       // flat candidate slots
  int n_tiles = 0;
  int max_halo_tiles = 0;
  int n_grid = 0;      // haloes
  int n_big = 0;       // haloes of more than 256 tiles
  bool fp64 = false;
  bool masses = false; // per-particle masses
  bool gas = false;
};

// The class's arrays, in one fixed order (sizing pass with G == NULL).
void grid_take(Bump& B, GridLaunch* G, const GridSizes& z) {
  const size_t es = z.fp64 ? 8 : 4;          // real
  const size_t v4 = 4 * es;                  // (w, r) or (v, m)
  const size_t as = z.fp64 ? 16 : 8;         // exact sum
  GridHaloState* st = B.take<GridHaloState>((size_t)z.n_grid);
  GridCtl* ctl = B.take<GridCtl>(1);
  char* rec = B.take<char>(z.nf * 2 * v4);
  char* ka = B.take<char>(z.nf * es);
  char* kb = B.take<char>(z.nf * es);
  uint32_t* va = B.take<uint32_t>(z.nf);
  uint32_t* vb = B.take<uint32_t>(z.nf);
  char* wr = B.take<char>(z.nf * v4);
  char* ms = B.take<char>(z.masses ? z.nf * es : 0);
  char* uth = B.take<char>(z.gas ? z.nf * es : 0);
  uint32_t* vx = B.take<uint32_t>(z.nf);
  char* mc = B.take<char>(z.nf * as);
  char* rcp = B.take<char>(z.nf * es);
  int2* trg = B.take<int2>((size_t)z.n_tiles);
  int* th = B.take<int>((size_t)z.n_tiles);
  int* ht0 = B.take<int>((size_t)z.n_grid + 1);
  int* big = B.take<int>((size_t)std::max(1, z.n_big));
  uint32_t* hist = B.take<uint32_t>((size_t)z.n_tiles * 256);
  uint32_t* dbase = B.take<uint32_t>((size_t)z.n_grid * 256);
  const size_t n_sub = (size_t)z.n_tiles * (GRID_TILE / GRID_SUB);
  char* agm = B.take<char>(2 * n_sub * as);
  char* agr = B.take<char>(2 * n_sub * as);
  int* agc = B.take<int>(2 * n_sub);
  char* prm_ = B.take<char>((size_t)z.n_tiles * as);
  char* prr = B.take<char>((size_t)z.n_tiles * as);
  long long* prc = B.take<long long>((size_t)z.n_tiles);
  int4* work = B.take<int4>(2 * n_sub);
  uint8_t* rmask = B.take<uint8_t>(32 * n_sub);
  AccSlot* tmv = B.take<AccSlot>(3 * (size_t)z.n_tiles);
  SkipRec* skip = B.take<SkipRec>(n_sub);
  if (!G) return;
  G->state = st; G->ctl = ctl; G->rec = rec; G->key_a = ka; G->key_b = kb; G->val_a = va; G->val_b = vb;
  G->wr = wr; G->ms = z.masses ? ms : nullptr; G->uth = z.gas ? uth : nullptr; G->val_x = vx; G->mc = mc;
  G->rc = rcp; G->tile_range = trg; G->tile_halo = th; G->halo_tile0 = ht0; G->big_halos = big;
  G->n_big = z.n_big; G->tile_hist = hist; G->digit_base = dbase;
  G->agg_m = agm; G->agg_r = agr; G->agg_c = agc; G->pre_m = prm_; G->pre_r = prr; G->pre_c = prc;
  G->work = work;
  G->rem_mask = rmask;
  G->tile_mv = tmv; G->skip = skip; G->max_halo_tiles = z.max_halo_tiles; G->n_halos = z.n_grid; G->n_flat = (long long)z.nf; G->n_tiles = z.n_tiles;
  G->fp64 = z.fp64 ? 1 : 0;
}

// Per-call device resets of the class's control words and halo states
// (before grid_prepare).
int grid_reset(const GridLaunch& G, cudaStream_t s) {
  AHF_CUDA(cudaMemsetAsync(G.state, 0, sizeof(GridHaloState) * (size_t)G.n_halos, s));
  AHF_CUDA(cudaMemsetAsync(G.ctl, 0, sizeof(GridCtl), s));
  AHF_CUDA(cudaMemsetAsync(&G.ctl->key_and, 0xff, sizeof(unsigned long long), s));
  return AHF_OK;
}

// Resident CTAs of the persistent pass on the context's device.
int grid_pass_ctas(ahf_ctx* c, bool fp64) {
  int& g = c->iter_grid[fp64 ? 1 : 0];
  if (g < 0) g = std::max(1, grid_iter_grid(c->device, fp64 ? 1 : 0));
  return g;
}

// Sort, iterate and finish the multi-CTA class (phases 8 to the end of the
// sort, 9 and 10).  The passes go out `chunk` at a time; the host reads the
// count of still-active haloes once per chunk (a pass with nothing left to
// do returns at once).
int run_grid(ahf_ctx* c, GridLaunch& G, const ahf_params* prm, cudaStream_t s, int chunk) {
  int rc;
  // the passes stage the stream through tensor copies (mixed mode, a uniform
  // mass, no gas) when the device takes them
  G.wait_limit = c->wait_limit;
  G.use_tma = 0;
  if (!G.fp64 && !G.ms && !G.uth) {
    if (c->tma_grid < 0) c->tma_grid = grid_tma_grid(c->device);
    G.tma_grid = c->tma_grid;
    if (G.tma_grid > 0 && grid_wr_map(G, (G.n_flat + 7) / 8)) G.use_tma = 1;
  }
  AHF_CUDA(cudaMemcpyAsync(c->flag_host, &G.ctl->key_or, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  AHF_CUDA(cudaStreamSynchronize(s));
  c->stats.host_syncs += 1;
  unsigned long long orb, andb;
  std::memcpy(&orb, c->flag_host, 8);
  std::memcpy(&andb, c->flag_host + 2, 8);
  AHF_CUDA(grid_sort(G, s, orb, andb));
  c->stats.launches += G.sort_launches;
  if ((rc = phase_end(c, PH_GRID_SORT, s))) return rc;
  if ((rc = phase_begin(c, PH_GRID_ITER, s, G.n_halos, G.n_flat))) return rc;
  for (int pass = 1; pass <= prm->max_iter;) {
    const int n = std::min(chunk, prm->max_iter - pass + 1);
    for (int i = 0; i < n; ++i) {
      AHF_CUDA(grid_iterate(G, pass++, s));
      c->stats.launches += 3;
      c->stats.grid_iterations += 1;
    }
    if (pass > prm->max_iter) break;
    AHF_CUDA(cudaMemcpyAsync(c->flag_host + 4, &G.ctl->work_n[pass & 1], sizeof(int), cudaMemcpyDeviceToHost, s));
    AHF_CUDA(cudaStreamSynchronize(s));
    c->stats.host_syncs += 1;
    if (c->flag_host[4] == 0) break;
  }
  if ((rc = phase_end(c, PH_GRID_ITER, s))) return rc;
  if ((rc = phase_begin(c, PH_GRID_FINISH, s, G.n_halos, G.n_flat))) return rc;
  AHF_CUDA(grid_finish(G, s));
  c->stats.launches += 3 + (G.rows.prof ? 1 : 0);
  return phase_end(c, PH_GRID_FINISH, s);
}

struct GridTables {
  std::vector<int2> tile_range;
  std::vector<int> tile_halo;
  std::vector<int> halo_tile0;
  std::vector<int> big;        // haloes of more than 256 tiles
};

void build_tiles(const Plan& P, int first, int n, GridTables& T) {
  T.tile_range.clear();
  T.tile_halo.clear();
  T.big.clear();
  T.halo_tile0.assign((size_t)n + 1, 0);
  for (int k = 0; k < n; ++k) {
    const HaloDev& d = P.hd[(size_t)first + k];
    T.halo_tile0[k] = (int)T.tile_range.size();
    for (long long o = 0; o < d.count; o += GRID_TILE) {
      const long long len = std::min<long long>(GRID_TILE, d.count - o);
      T.tile_range.push_back(make_int2((int)(d.gbase + o), (int)len));
      T.tile_halo.push_back(k);
    }
    if ((int)T.tile_range.size() - T.halo_tile0[k] > 256) T.big.push_back(k);
  }
  T.halo_tile0[n] = (int)T.tile_range.size();
}

int profile_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                 const int64_t* member_idx, const ahf_params* prm, const ahf_result* res, const int64_t* bound_idx,
                 int32_t n_bins, double r_min_frac, double* prof, cudaStream_t s,
                 const std::vector<char>* include = nullptr);

// Outputs of the host-buffer entry point that each class pushes to the
// caller's page-locked buffers as soon as its kernel is done
// (AHF_OPT_HOST_DIRECT 2), while the other classes still run: the device
// arrays the kernels wrote and the buffers' mapped device addresses.
struct HostPush {
  const ahf_result* res;     // device records (each halo's n_bound)
  const long long* bi;       // device bound lists
  long long* h_bi;
  const char* phi;           // device phi (NULL: none)
  char* h_phi;
  int phi_es;                // 4 or 8
  const int* ri;             // device removal iterations (NULL: none)
  int* h_ri;
};

// Copy each halo's bound list and phi (its first n_bound slots) and its
// removal iterations (all its slots) from device memory to the mapped host
// buffers; CTA (k, j) takes the j-th of gridDim.y shares of halo k.
// Consecutive threads write consecutive slots, so the host link carries
// whole lines.
__global__ void __launch_bounds__(256) push_slots(HostPush a, const HaloDev* __restrict__ hd) {
  const HaloDev& H = hd[blockIdx.x];
  const long long o = H.offset;
  const long long nb = a.res[H.index].n_bound;
  const long long per_b = ((nb + gridDim.y - 1) / gridDim.y + 255) & ~255ll;
  const long long lo = (long long)blockIdx.y * per_b, hi = nb < lo + per_b ? nb : lo + per_b;
  for (long long i = lo + threadIdx.x; i < hi; i += 256) {
    a.h_bi[o + i] = a.bi[o + i];
    if (a.phi) {
      if (a.phi_es == 8) ((double*)a.h_phi)[o + i] = ((const double*)a.phi)[o + i];
      else ((float*)a.h_phi)[o + i] = ((const float*)a.phi)[o + i];
    }
  }
  if (a.ri) {
    const long long n = H.count;
    const long long per = ((n + gridDim.y - 1) / gridDim.y + 255) & ~255ll;
    const long long l2 = (long long)blockIdx.y * per, h2 = n < l2 + per ? n : l2 + per;
    for (long long i = l2 + threadIdx.x; i < h2; i += 256) a.h_ri[o + i] = a.ri[o + i];
  }
}

// The push of n haloes (largest count maxc) on stream s.
cudaError_t launch_push(const HostPush& a, const HaloDev* hd, int n, long long maxc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int split = (int)std::min<long long>(256, std::max<long long>(1, (maxc + 8191) / 8192));
  push_slots<<<dim3((unsigned)n, (unsigned)split), 256, 0, s>>>(a, hd);
  return cudaGetLastError();
}

// Unbinding of a batch; with prof != NULL also the profile rows.  The warp
// and single-CTA variants form the rows from the bound set they hold on chip;
// haloes of the cluster and multi-CTA classes get theirs from the profile
// kernels afterwards.
int unbind_pass(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx, void* phi,
                int32_t* removed_iter, cudaStream_t s, int32_t n_bins = 0, double r_min_frac = 0.0,
                double* prof = nullptr, const HostPush* push = nullptr) {
  int rc = validate(p, halos, n_halos, prm, out, bound_idx);
  if (rc) return rc;
  if (prof && (n_bins < 1 || n_bins > profile_max_bins()))
    return fail(AHF_ERR_INVALID, "n_bins must be in [1, %d]", profile_max_bins());
  if (prof && !(r_min_frac > 0.0 && r_min_frac < 1.0)) return fail(AHF_ERR_INVALID, "r_min_frac must be in (0, 1)");
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  if ((rc = validate_slots(halos, n_halos, n_slots, member_idx != nullptr))) return rc;
  if (n_halos == 0) return AHF_OK;
  Plan P;
  if ((rc = make_plan(c, p, halos, n_halos, prm, P))) return rc;
  reset_stats(c);
  // variants 0..3 form profile rows themselves, the clusters (4..6) too when
  // the bin count fits their exchange record
  const int FUSED_MAX = n_bins <= 128 ? NV - 1 : 3;
  int n_onchip = 0;
  for (int v = 0; v < NV; ++v) n_onchip += P.n_class[v];
  const int n_grid = P.n_class[NV];
  if (P.grid_flat >= (1ll << 31)) return fail(AHF_ERR_INVALID, "multi-CTA class above 2^31 candidates");
  GridTables T;
  if (n_grid) build_tiles(P, n_onchip, n_grid, T);
  const int n_tiles = (int)T.tile_range.size();
  const size_t nf = (size_t)P.grid_flat;
  const bool fp64 = prm->precision == AHF_PREC_FP64;
  GridSizes gz;
  gz.nf = nf; gz.n_tiles = n_tiles; gz.n_grid = n_grid; gz.n_big = (int)T.big.size(); gz.fp64 = fp64;
  for (int k = 0; k < n_grid; ++k)
    gz.max_halo_tiles = std::max(gz.max_halo_tiles, T.halo_tile0[(size_t)k + 1] - T.halo_tile0[(size_t)k]);
  gz.masses = p->m != nullptr; gz.gas = p->u_th != nullptr;

  // workspace layout (must match the Bump sequence below)
  double* dfac = nullptr;
  float* dfacf = nullptr;
  float4* drec = nullptr;
  auto layout = [&](Bump& B, GridLaunch* G) {
    HaloDev* hd = B.take<HaloDev>((size_t)n_halos);
    int* queues = B.take<int>(16);
    double* fac = B.take<double>(prof ? 3 * (size_t)n_bins : 0);
    float* facf = B.take<float>(prof ? 3 * (size_t)n_bins : 0);
    float4* rec = B.take<float4>(2 * (size_t)P.onchip_flat);
    if (G) { dfac = fac; dfacf = facf; drec = P.onchip_flat ? rec : nullptr; }
    if (G) G->halos = hd + n_onchip;
    if (n_grid) grid_take(B, G, gz);
    return hd;
  };
  Bump sizing{nullptr, 0, 0};
  layout(sizing, nullptr);
  if ((rc = ensure_workspace(c, sizing.used + 4096))) return rc;
  const size_t pin_need = sizeof(HaloDev) * (size_t)n_halos + 1024 + (prof ? 36 * (size_t)n_bins + 512 : 0) +
                          (sizeof(int2) + sizeof(int)) * (size_t)n_tiles + 256 + sizeof(int) * ((size_t)n_grid + 1) + 256 +
                          sizeof(int) * T.big.size() + 256;
  if ((rc = begin_call(c, s))) return rc;
  Bump B{c->ws, 0, c->ws_bytes};
  GridLaunch G{};
  HaloDev* hd = layout(B, &G);
  int* queues = reinterpret_cast<int*>(reinterpret_cast<char*>(hd) + align_up(sizeof(HaloDev) * (size_t)n_halos, 256));
  char* pin = nullptr;
  if ((rc = pin_acquire(c, pin_need, &pin))) return rc;
  size_t po = 0;
  auto stage = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    po = align_up(po, 256);
    std::memcpy(pin + po, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, pin + po, bytes, cudaMemcpyHostToDevice, s);
    po += bytes;
    return e;
  };
  {
    // descriptors, zeroed queue counters and the bin tables sit back to back
    // in the workspace: one copy of the same image from pinned memory
    char* d0 = reinterpret_cast<char*>(hd);
    const size_t qo = (size_t)(reinterpret_cast<char*>(queues) - d0);
    size_t span = qo + 16 * sizeof(int);
    std::memcpy(pin, P.hd.data(), sizeof(HaloDev) * (size_t)n_halos);
    std::memset(pin + sizeof(HaloDev) * (size_t)n_halos, 0, span - sizeof(HaloDev) * (size_t)n_halos);
    if (prof) {
      std::vector<double> tab(3 * (size_t)n_bins);
      profile_bin_tables(n_bins, r_min_frac, tab.data());
      const size_t fo = (size_t)(reinterpret_cast<char*>(dfac) - d0);
      const size_t ffo = (size_t)(reinterpret_cast<char*>(dfacf) - d0);
      std::memset(pin + span, 0, fo - span);
      std::memcpy(pin + fo, tab.data(), sizeof(double) * tab.size());
      std::memset(pin + fo + sizeof(double) * tab.size(), 0, ffo - fo - sizeof(double) * tab.size());
      float* tf = reinterpret_cast<float*>(pin + ffo);
      for (size_t k = 0; k < tab.size(); ++k) tf[k] = (float)tab[k];
      span = ffo + sizeof(float) * tab.size();
    }
    AHF_CUDA(cudaMemcpyAsync(d0, pin, span, cudaMemcpyHostToDevice, s));
    po = span;
    // the counters are zeroed once more by a kernel: with the graph launched
    // right behind the copy, on a stream still busy with the caller's input
    // copies, the batch started ~150 us late (host-buffer call 0.88 against
    // 0.71 ms on the 2,000-halo batch)
    AHF_CUDA(cudaMemsetAsync(queues, 0, 16 * sizeof(int), s));
  }

  OutputsDev O;
  std::memset(&O, 0, sizeof O);
  O.res = out; O.bound_idx = (long long*)bound_idx; O.phi = phi; O.removed_iter = removed_iter;
  O.member_idx = (const long long*)member_idx; O.n_slots = n_slots; O.err = c->err_dev;
  const ParticlesDev pd = to_dev(p);
  const ParamsDev prd = to_dev(prm);

  if (n_grid) {
    AHF_CUDA(stage(G.tile_range, T.tile_range.data(), sizeof(int2) * (size_t)n_tiles));
    AHF_CUDA(stage(G.tile_halo, T.tile_halo.data(), sizeof(int) * (size_t)n_tiles));
    AHF_CUDA(stage(G.halo_tile0, T.halo_tile0.data(), sizeof(int) * ((size_t)n_grid + 1)));
    AHF_CUDA(stage(G.big_halos, T.big.data(), sizeof(int) * T.big.size()));
    if ((rc = grid_reset(G, s))) return rc;
    G.p = pd; G.frame = P.frame; G.prm = prd; G.out = O;
    G.iter_grid = grid_pass_ctas(c, fp64);
    // profile rows of this class from its final pass
    G.rows.prof = prof;
    G.rows.factor = dfac;
    G.rows.factor_f = dfacf;
    G.rows.n_bins = n_bins;
    if ((rc = phase_begin(c, PH_GRID_SORT, s, n_grid, (long long)nf))) return rc;
    AHF_CUDA(grid_prepare(G, s));
    c->stats.launches += 2;
  }
  if ((rc = pin_release(c, s))) return rc;
  if (c->trace) {
    if (c->trace_cap < n_halos) {
      if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
      if (c->trace_dev) cudaFree(c->trace_dev);
      c->trace_dev = nullptr;
      c->trace_cap = 0;
      if (cudaMalloc(&c->trace_dev, sizeof(long long) * AHF_TRACE_FIELDS * (size_t)n_halos) != cudaSuccess) {
        cudaGetLastError();
        return fail(AHF_ERR_NOMEM, "trace buffer");
      }
      c->trace_cap = n_halos;
    }
    AHF_CUDA(cudaMemsetAsync(c->trace_dev, 0, sizeof(long long) * AHF_TRACE_FIELDS * (size_t)n_halos, s));
    c->trace_n = n_halos;
  }
  // the on-chip variants run on side streams, largest first, concurrently
  // with the multi-CTA class on the caller's stream
  struct VLaunch {
    int v, grid, n;
    long long cands;
    OnchipLaunch L;
  };
  std::vector<VLaunch> vl;
  int first_of[NV];
  for (int v = 0, f = 0; v < NV; ++v) { first_of[v] = f; f += P.n_class[v]; }
  // launch order (the block scheduler serves earlier launches first): the
  // clusters (largest haloes) first, then the single-CTA variants of 8k and
  // 4k slots, then the warp variant, whose haloes run longer than the 1k
  // variant's, then that one
  constexpr int kOrder[NV] = {7, 6, 5, 4, 3, 2, 0, 1};
  for (int oi = 0; oi < NV; ++oi) {
    const int v = kOrder[oi];
    const int n = P.n_class[v];
    if (n == 0) continue;
    VLaunch x;
    std::memset(&x, 0, sizeof x);        // padding too: the bytes form the graph key
    x.v = v;
    x.n = n;
    OnchipLaunch& L = x.L;
    L.p = pd; L.frame = P.frame; L.prm = prd; L.out = O;
    L.halos = hd + first_of[v]; L.n_halos = n; L.queue = queues + v;
    L.rows.prof = (prof && v <= FUSED_MAX) ? prof : nullptr;
    L.rows.factor = dfac;
    L.rows.factor_f = dfacf;
    L.rows.n_bins = n_bins;
    L.trace = c->trace ? c->trace_dev : nullptr;
    L.variant = v;
    L.rec = drec;
    for (int k = 0; k < n; ++k) x.cands += P.hd[(size_t)first_of[v] + k].count;
    x.grid = (int)std::min<long long>(variant_grid_for(v, n), c->variant_grid[v]);
    vl.push_back(x);
  }
  auto enqueue_onchip = [&](cudaStream_t o, bool join) -> int {
    if (c->serial) {                     // one class after another on the caller's stream
      for (const VLaunch& x : vl) {
        int prc;
        if ((prc = phase_begin(c, x.v, o, 0, 0))) return prc;
        AHF_CUDA(launch_variant(x.L, x.v, x.grid, o));
        if ((prc = phase_end(c, x.v, o))) return prc;
        if (push) AHF_CUDA(launch_push(*push, x.L.halos, x.n, P.hd[(size_t)first_of[x.v]].count, o));
      }
      return AHF_OK;
    }
    AHF_CUDA(cudaEventRecord(c->fork, o));
    for (const VLaunch& x : vl) {
      AHF_CUDA(cudaStreamWaitEvent(c->side[x.v], c->fork, 0));
      int prc;
      if ((prc = phase_begin(c, x.v, c->side[x.v], 0, 0))) return prc;
      AHF_CUDA(launch_variant(x.L, x.v, x.grid, c->side[x.v]));
      if ((prc = phase_end(c, x.v, c->side[x.v]))) return prc;
      if (push) AHF_CUDA(launch_push(*push, x.L.halos, x.n, P.hd[(size_t)first_of[x.v]].count, c->side[x.v]));
      AHF_CUDA(cudaEventRecord(c->join[x.v], c->side[x.v]));
    }
    if (join)
      for (const VLaunch& x : vl) AHF_CUDA(cudaStreamWaitEvent(o, c->join[x.v], 0));
    return AHF_OK;
  };
  for (const VLaunch& x : vl) {
    c->stats.launches += push ? 2 : 1;
    c->phase_used[x.v] = true;
    c->stats.phase_halos[x.v] += x.n;
    c->stats.phase_candidates[x.v] += x.cands;
  }
  // a batch of on-chip haloes only can run as a CUDA graph, replayed while
  // the launch parameters repeat (the descriptors staged above are inputs
  // of the graph's kernels, not part of it); with outputs pushed to host
  // buffers, their addresses and each class's push grid are parameters too
  if (c->graphs && !c->timing && n_grid == 0 && !vl.empty()) {
    std::vector<unsigned char> key(vl.size() * sizeof(VLaunch));
    std::memcpy(key.data(), vl.data(), key.size());
    if (push) {
      auto put = [&](const void* v, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(v);
        key.insert(key.end(), b, b + n);
      };
      const void* ptrs[7] = {push->res, push->bi, push->h_bi, push->phi, push->h_phi, push->ri, push->h_ri};
      put(ptrs, sizeof ptrs);
      put(&push->phi_es, sizeof push->phi_es);
      for (const VLaunch& x : vl) put(&P.hd[(size_t)first_of[x.v]].count, sizeof(long long));
    }
    if (!c->graph_exec || key != c->graph_key) {
      if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
      c->graph_key.clear();
      // captured on the context's own stream (the caller's may be the legacy
      // default stream, which cannot be captured); launched on the caller's
      AHF_CUDA(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeRelaxed));
      const int erc = enqueue_onchip(c->capture, true);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(c->capture, &g);
      if (erc != AHF_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return erc != AHF_OK ? erc : fail(AHF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
      }
      const cudaError_t ie = cudaGraphInstantiate(&c->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        c->graph_exec = nullptr;
        cudaGetLastError();
        return fail(AHF_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ie));
      }
      c->graph_key = key;
      c->stats.graph_captures += 1;
    }
    AHF_CUDA(cudaGraphLaunch(c->graph_exec, s));
    c->stats.graph_launches += 1;
  } else {
    if ((rc = enqueue_onchip(s, false))) return rc;
    if (n_grid) {
      if ((rc = run_grid(c, G, prm, s, c->pass_chunk))) return rc;
      if (push) {
        AHF_CUDA(launch_push(*push, hd + n_onchip, n_grid, P.hd[(size_t)n_onchip].count, s));
        c->stats.launches += 1;
      }
    }
    if (!c->serial)
      for (const VLaunch& x : vl) AHF_CUDA(cudaStreamWaitEvent(s, c->join[x.v], 0));
  }
  if ((rc = end_call(c, s))) return rc;
  if (prof) {
    // rows of the haloes the fused variants did not cover
    std::vector<char> rest((size_t)n_halos, 0);
    bool any = false;
    int64_t first = 0;
    for (int v = 0; v <= NV; ++v) {
      for (int k = 0; k < P.n_class[v]; ++k)
        if (v > FUSED_MAX && v < NV) { rest[(size_t)P.hd[(size_t)(first + k)].index] = 1; any = true; }
      first += P.n_class[v];
    }
    if (any) return profile_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, n_bins, r_min_frac, prof, s,
                                 &rest);
    // the profile phase then covers the fused rows only
    c->stats.phase_halos[PH_PROFILE] = 0;
  }
  return AHF_OK;
}


int profile_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                 const int64_t* member_idx, const ahf_params* prm, const ahf_result* res, const int64_t* bound_idx,
                 int32_t n_bins, double r_min_frac, double* prof, cudaStream_t s, const std::vector<char>* include) {
  int rc = validate(p, halos, n_halos, prm, res, bound_idx);
  if (rc) return rc;
  if (n_halos > 0 && !prof) return fail(AHF_ERR_INVALID, "prof must not be NULL");
  if (n_bins < 1 || n_bins > profile_max_bins()) return fail(AHF_ERR_INVALID, "n_bins must be in [1, %d]", profile_max_bins());
  if (!(r_min_frac > 0.0 && r_min_frac < 1.0)) return fail(AHF_ERR_INVALID, "r_min_frac must be in (0, 1)");
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  if ((rc = validate_slots(halos, n_halos, n_slots, member_idx != nullptr))) return rc;
  if (n_halos == 0) return AHF_OK;
  Plan P;
  if ((rc = make_plan(c, p, halos, n_halos, prm, P))) return rc;
  // descriptors in the caller's order (make_plan reorders by class)
  std::vector<HaloDev> hd((size_t)n_halos);
  for (const HaloDev& d : P.hd) hd[(size_t)d.index] = d;
  std::vector<int> chunk_halo, halo_chunk0((size_t)n_halos + 1);
  std::vector<long long> chunk_start;
  for (int64_t h = 0; h < n_halos; ++h) {
    halo_chunk0[(size_t)h] = (int)chunk_halo.size();
    if (include && !(*include)[(size_t)h]) continue;
    // a halo with no candidates still needs one chunk to write its zero rows
    const long long cnt = std::max<long long>(halos[h].count, 1);
    for (long long o = 0; o < cnt; o += PROFILE_CHUNK) {
      chunk_halo.push_back((int)h);
      chunk_start.push_back(o);
    }
  }
  halo_chunk0[(size_t)n_halos] = (int)chunk_halo.size();
  const int n_chunks = (int)chunk_halo.size();
  int n_multi = 0;
  for (int64_t h = 0; h < n_halos; ++h) n_multi += halo_chunk0[(size_t)h + 1] - halo_chunk0[(size_t)h] > 1;
  std::vector<double> factor(3 * (size_t)n_bins);
  profile_bin_tables(n_bins, r_min_frac, factor.data());
  double* dfac = nullptr;
  float* dfacf = nullptr;
  auto layout = [&](Bump& B, ProfileLaunch* L, int** h0) {
    HaloDev* d = B.take<HaloDev>((size_t)n_halos);
    int* ch = B.take<int>((size_t)n_chunks + 1);
    long long* cs = B.take<long long>((size_t)n_chunks + 1);
    int* hc0 = B.take<int>((size_t)n_halos + 1);
    double* fac = B.take<double>(3 * (size_t)n_bins);
    float* facf = B.take<float>(3 * (size_t)n_bins);
    long long* acc = B.take<long long>((size_t)n_chunks * (2 + 2 * (size_t)n_bins) + 1);
    if (L) {
      L->halos = d; L->chunk_halo = ch; L->chunk_start = cs; L->chunk_acc = acc; *h0 = hc0;
      dfac = fac;
      dfacf = facf;
    }
  };
  Bump sizing{nullptr, 0, 0};
  layout(sizing, nullptr, nullptr);
  if ((rc = ensure_workspace(c, sizing.used + 4096))) return rc;
  if ((rc = begin_call(c, s))) return rc;
  Bump B{c->ws, 0, c->ws_bytes};
  ProfileLaunch L{};
  int* hc0 = nullptr;
  layout(B, &L, &hc0);
  char* pin = nullptr;
  if ((rc = pin_acquire(c, sizing.used + 4096, &pin))) return rc;
  size_t po = 0;
  auto stage = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    po = align_up(po, 256);
    std::memcpy(pin + po, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, pin + po, bytes, cudaMemcpyHostToDevice, s);
    po += bytes;
    return e;
  };
  AHF_CUDA(stage((void*)L.halos, hd.data(), sizeof(HaloDev) * (size_t)n_halos));
  AHF_CUDA(stage(L.chunk_halo, chunk_halo.data(), sizeof(int) * (size_t)n_chunks));
  AHF_CUDA(stage(L.chunk_start, chunk_start.data(), sizeof(long long) * (size_t)n_chunks));
  AHF_CUDA(stage(hc0, halo_chunk0.data(), sizeof(int) * ((size_t)n_halos + 1)));
  AHF_CUDA(stage(dfac, factor.data(), sizeof(double) * factor.size()));
  const std::vector<float> factor_f(factor.begin(), factor.end());
  AHF_CUDA(stage(dfacf, factor_f.data(), sizeof(float) * factor_f.size()));
  if ((rc = pin_release(c, s))) return rc;
  L.edge_factor = dfac;
  L.edge_factor_f = dfacf;
  L.n_multi = n_multi;
  L.p = to_dev(p);
  L.frame = P.frame;
  L.prm = to_dev(prm);
  L.out.err = c->err_dev;
  L.out.member_idx = (const long long*)member_idx;
  L.n_halos = (int)n_halos;
  L.res = res;
  L.bound_idx = (const long long*)bound_idx;
  L.n_bins = n_bins;
  L.r_min_frac = r_min_frac;
  L.prof = prof;
  L.n_chunks = n_chunks;
  c->phase_used[PH_PROFILE] = false;
  c->stats.phase_ms[PH_PROFILE] = -1.0;
  c->stats.phase_halos[PH_PROFILE] = 0;
  c->stats.phase_candidates[PH_PROFILE] = 0;
  if ((rc = phase_begin(c, PH_PROFILE, s, n_halos, (long long)n_chunks * PROFILE_CHUNK))) return rc;
  AHF_CUDA(launch_profile(L, hc0, s));
  c->stats.launches += (n_chunks > 0 ? 1 : 0) + (n_multi > 0 ? 1 : 0);
  if ((rc = phase_end(c, PH_PROFILE, s))) return rc;
  return end_call(c, s);
}

// One halo at a time: the multi-CTA kernels on a single halo, with a host
// synchronisation on every iteration's change flag (the plain launch form).
int plain_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
               const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx, void* phi,
               int32_t* removed_iter, cudaStream_t s) {
  int rc = validate(p, halos, n_halos, prm, out, bound_idx);
  if (rc) return rc;
  if (prm->variant & AHF_VAR_RETRUNCATE) return fail(AHF_ERR_INVALID, "the plain path has no AHF_VAR_RETRUNCATE");
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  if ((rc = validate_slots(halos, n_halos, n_slots, member_idx != nullptr))) return rc;
  if (n_halos == 0) return AHF_OK;
  Plan P;
  if ((rc = make_plan(c, p, halos, n_halos, prm, P))) return rc;
  long long maxc = 1;
  for (const HaloDev& d : P.hd) maxc = std::max(maxc, d.count);
  const size_t nf = (size_t)((maxc + 7) & ~7ll);
  const int max_tiles = (int)((maxc + GRID_TILE - 1) / GRID_TILE);
  GridSizes gz;
  gz.nf = nf; gz.n_tiles = max_tiles; gz.n_grid = 1; gz.n_big = max_tiles > 256 ? 1 : 0;
  gz.max_halo_tiles = max_tiles;
  gz.fp64 = prm->precision == AHF_PREC_FP64; gz.masses = p->m != nullptr; gz.gas = p->u_th != nullptr;
  auto layout = [&](Bump& B, GridLaunch* G) {
    HaloDev* hd = B.take<HaloDev>(1);
    if (G) G->halos = hd;
    grid_take(B, G, gz);
  };
  Bump sizing{nullptr, 0, 0};
  layout(sizing, nullptr);
  if ((rc = ensure_workspace(c, sizing.used + 4096))) return rc;
  const size_t pin_need = sizeof(HaloDev) + (sizeof(int2) + sizeof(int)) * (size_t)max_tiles + 2048;
  if ((rc = begin_call(c, s))) return rc;
  Bump B{c->ws, 0, c->ws_bytes};
  GridLaunch G{};
  layout(B, &G);
  OutputsDev O;
  std::memset(&O, 0, sizeof O);
  O.res = out; O.bound_idx = (long long*)bound_idx; O.phi = phi; O.removed_iter = removed_iter;
  O.member_idx = (const long long*)member_idx; O.n_slots = n_slots; O.err = c->err_dev;
  G.p = to_dev(p); G.frame = P.frame; G.prm = to_dev(prm); G.out = O;
  G.iter_grid = grid_pass_ctas(c, gz.fp64);
  reset_stats(c);
  for (const HaloDev& d0 : P.hd) {
    HaloDev d = d0;
    d.gbase = 0;
    // one halo: tile table
    std::vector<int2> tr;
    std::vector<int> th;
    for (long long o = 0; o < d.count; o += GRID_TILE) {
      tr.push_back(make_int2((int)o, (int)std::min<long long>(GRID_TILE, d.count - o)));
      th.push_back(0);
    }
    const int ht0[2] = {0, (int)tr.size()};
    const int big0 = 0;
    G.n_tiles = (int)tr.size();
    G.n_flat = d.count;
    G.n_big = G.n_tiles > 256 ? 1 : 0;
    char* pin = nullptr;
    if ((rc = pin_acquire(c, pin_need, &pin))) return rc;
    size_t po = 0;
    auto stage = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
      if (bytes == 0) return cudaSuccess;
      po = align_up(po, 256);
      std::memcpy(pin + po, src, bytes);
      cudaError_t e = cudaMemcpyAsync(dst, pin + po, bytes, cudaMemcpyHostToDevice, s);
      po += bytes;
      return e;
    };
    AHF_CUDA(stage(G.halos, &d, sizeof(HaloDev)));
    AHF_CUDA(stage(G.tile_range, tr.data(), sizeof(int2) * tr.size()));
    AHF_CUDA(stage(G.tile_halo, th.data(), sizeof(int) * th.size()));
    AHF_CUDA(stage(G.halo_tile0, ht0, sizeof(ht0)));
    AHF_CUDA(stage(G.big_halos, &big0, sizeof(int)));
    if ((rc = pin_release(c, s))) return rc;
    if ((rc = grid_reset(G, s))) return rc;
    if (G.n_tiles == 0) {
      // no candidates: an empty record
      ahf_result R{};
      R.status = AHF_HALO_EMPTY;
      R.k_vir = -1;
      AHF_CUDA(cudaMemcpyAsync(out + d.index, &R, sizeof(R), cudaMemcpyHostToDevice, s));
      AHF_CUDA(cudaStreamSynchronize(s));
      continue;
    }
    if ((rc = phase_begin(c, PH_GRID_SORT, s, 1, d.count))) return rc;
    AHF_CUDA(grid_prepare(G, s));
    c->stats.launches += 2;
    // the plain form reads the change flag after every pass
    if ((rc = run_grid(c, G, prm, s, 1))) return rc;
  }
  return end_call(c, s);
}

// Host-memory form: stage the inputs in a device buffer, run, copy back.
int props_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos, const int64_t* member_idx,
               const ahf_params* prm, const ahf_result* res, const int64_t* bound_idx, const void* phi, double* props,
               cudaStream_t s) {
  int rc = validate(p, halos, n_halos, prm, res, bound_idx);
  if (rc) return rc;
  if (n_halos > 0 && (!phi || !props)) return fail(AHF_ERR_INVALID, "phi and props must not be NULL");
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  if ((rc = validate_slots(halos, n_halos, n_slots, member_idx != nullptr))) return rc;
  if (n_halos == 0) return AHF_OK;
  // descriptors in the caller's order; chunks over each halo's slots (an
  // upper bound of its bound list; chunks past the list do no work)
  std::vector<HaloDev> hd((size_t)n_halos);
  for (int64_t h = 0; h < n_halos; ++h) fill_halo_dev(halos[h], p->coord_type, prm->box, (int)h, hd[(size_t)h]);
  std::vector<int> chunk_halo, halo_chunk0((size_t)n_halos + 1);
  std::vector<long long> chunk_start;
  for (int64_t h = 0; h < n_halos; ++h) {
    halo_chunk0[(size_t)h] = (int)chunk_halo.size();
    for (long long o = 0; o < halos[h].count; o += PROPS_CHUNK) {
      chunk_halo.push_back((int)h);
      chunk_start.push_back(o);
    }
  }
  halo_chunk0[(size_t)n_halos] = (int)chunk_halo.size();
  const int n_chunks = (int)chunk_halo.size();
  PropsLaunch L{};
  int* hc0 = nullptr;
  auto layout = [&](Bump& B, bool set) {
    HaloDev* d = B.take<HaloDev>((size_t)n_halos);
    int* ch = B.take<int>((size_t)n_chunks + 1);
    long long* cs = B.take<long long>((size_t)n_chunks + 1);
    int* h0 = B.take<int>((size_t)n_halos + 1);
    double* part = B.take<double>((size_t)n_chunks * PROPS_PART + 1);
    if (set) { L.halos = d; L.chunk_halo = ch; L.chunk_start = cs; hc0 = h0; L.part = part; }
  };
  Bump sizing{nullptr, 0, 0};
  layout(sizing, false);
  if ((rc = ensure_workspace(c, sizing.used + 4096))) return rc;
  if ((rc = begin_call(c, s))) return rc;
  Bump B{c->ws, 0, c->ws_bytes};
  layout(B, true);
  char* pin = nullptr;
  if ((rc = pin_acquire(c, sizing.used + 4096, &pin))) return rc;
  size_t po = 0;
  auto stage = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    po = align_up(po, 256);
    std::memcpy(pin + po, src, bytes);
    cudaError_t e = cudaMemcpyAsync(dst, pin + po, bytes, cudaMemcpyHostToDevice, s);
    po += bytes;
    return e;
  };
  AHF_CUDA(stage((void*)L.halos, hd.data(), sizeof(HaloDev) * (size_t)n_halos));
  AHF_CUDA(stage((void*)L.chunk_halo, chunk_halo.data(), sizeof(int) * (size_t)n_chunks));
  AHF_CUDA(stage((void*)L.chunk_start, chunk_start.data(), sizeof(long long) * (size_t)n_chunks));
  AHF_CUDA(stage(hc0, halo_chunk0.data(), sizeof(int) * ((size_t)n_halos + 1)));
  if ((rc = pin_release(c, s))) return rc;
  L.p = to_dev(p);
  L.frame.box = prm->box;
  L.G = prm->G;
  L.H = prm->H;
  L.n_halos = (int)n_halos;
  L.res = res;
  L.bound_idx = (const long long*)bound_idx;
  L.phi = phi;
  L.phi_f64 = prm->precision == AHF_PREC_FP64 ? 1 : 0;
  L.halo_chunk0 = hc0;
  L.n_chunks = n_chunks;
  L.props = props;
  AHF_CUDA(launch_properties(L, s));
  reset_stats(c);
  c->stats.launches = (n_chunks > 0 ? 2 : 0) + 1;
  return end_call(c, s);
}

int match_impl(ahf_ctx* c, int64_t n_ids, const int64_t* ids_a, const int64_t* off_a, const int64_t* cnt_a,
               int64_t n_a, const int64_t* ids_b, const int64_t* off_b, const int64_t* cnt_b, int64_t n_b,
               int64_t* best, int64_t* shared, double* xi, cudaStream_t s) {
  if (n_ids < 0 || n_a < 0 || n_b < 0) return fail(AHF_ERR_INVALID, "negative size");
  if (n_ids >= ((int64_t)1 << 40)) return fail(AHF_ERR_INVALID, "n_ids above 2^40");
  if (n_a > 0x7fffffff || n_b > 0x7fffffff) return fail(AHF_ERR_INVALID, "catalogue above 2^31-1 haloes");
  if (n_a > 0 && (!ids_a || !off_a || !cnt_a || !best || !shared || !xi))
    return fail(AHF_ERR_INVALID, "first catalogue or outputs NULL");
  if (n_b > 0 && (!ids_b || !off_b || !cnt_b)) return fail(AHF_ERR_INVALID, "second catalogue NULL");
  if (n_a == 0) return AHF_OK;
  Bump sizing{nullptr, 0, 0};
  sizing.take<int>((size_t)std::max<int64_t>(n_ids, 1));
  int rc;
  if ((rc = ensure_workspace(c, sizing.used + 4096))) return rc;
  if ((rc = begin_call(c, s))) return rc;
  Bump B{c->ws, 0, c->ws_bytes};
  MatchLaunch L{};
  L.label = B.take<int>((size_t)std::max<int64_t>(n_ids, 1));
  if (n_ids) AHF_CUDA(cudaMemsetAsync(L.label, 0xff, sizeof(int) * (size_t)n_ids, s));
  L.n_ids = n_ids;
  L.ids_a = (const long long*)ids_a; L.off_a = (const long long*)off_a; L.cnt_a = (const long long*)cnt_a;
  L.n_a = (int)n_a;
  L.ids_b = (const long long*)ids_b; L.off_b = (const long long*)off_b; L.cnt_b = (const long long*)cnt_b;
  L.n_b = (int)n_b;
  L.err = c->err_dev;
  L.best = (long long*)best; L.shared = (long long*)shared; L.xi = xi;
  AHF_CUDA(launch_match(L, s));
  reset_stats(c);
  c->stats.launches = (n_b > 0 ? 1 : 0) + 1;
  return end_call(c, s);
}

// Depth of every halo in the forest parent describes; -1 on a bad index or a
// cycle.
int forest_depths(const int64_t* parent, int64_t n, std::vector<int>& depth) {
  depth.assign((size_t)n, -1);
  std::vector<int64_t> chain;
  for (int64_t h = 0; h < n; ++h) {
    chain.clear();
    int64_t k = h;
    while (k >= 0 && depth[(size_t)k] < 0) {
      if (parent[k] < -1 || parent[k] >= n || (int64_t)chain.size() > n) return -1;
      chain.push_back(k);
      k = parent[k];
    }
    int base = k < 0 ? -1 : depth[(size_t)k];
    for (size_t i = chain.size(); i-- > 0;) depth[(size_t)chain[i]] = ++base;
  }
  return 0;
}

// The unbinding, with AHF_VAR_RETRUNCATE as a second pass over each halo's
// first-pass bound particles within its r_vir (the first pass's bound lists
// become the second pass's member lists).
int unbind_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx, void* phi,
                int32_t* removed_iter, cudaStream_t s, int32_t n_bins = 0, double r_min_frac = 0.0,
                double* prof = nullptr, const HostPush* push = nullptr) {
  if (!prm || !(prm->variant & AHF_VAR_RETRUNCATE))
    return unbind_pass(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter, s, n_bins,
                       r_min_frac, prof, push);
  ahf_params p1 = *prm;
  p1.variant &= ~AHF_VAR_RETRUNCATE;
  int rc = unbind_pass(c, p, halos, n_halos, member_idx, &p1, out, bound_idx, phi, removed_iter, s);
  if (rc || n_halos == 0) return rc;
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  // the first pass's bound lists (particle indices) as member lists
  const size_t need = sizeof(int64_t) * (size_t)std::max<int64_t>(n_slots, 1);
  if (need > c->aux_bytes) {
    if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
    if (c->aux) cudaFree(c->aux);
    c->aux = nullptr;
    c->aux_bytes = 0;
    if (cudaMalloc(&c->aux, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(AHF_ERR_NOMEM, "second-pass member lists (%zu bytes)", need);
    }
    c->aux_bytes = need;
  }
  int64_t* members = (int64_t*)c->aux;
  std::vector<ahf_result> r1((size_t)n_halos);
  if (n_slots) AHF_CUDA(cudaMemcpyAsync(members, bound_idx, (size_t)n_slots * 8, cudaMemcpyDeviceToDevice, s));
  AHF_CUDA(cudaMemcpyAsync(r1.data(), out, sizeof(ahf_result) * (size_t)n_halos, cudaMemcpyDeviceToHost, s));
  AHF_CUDA(cudaStreamSynchronize(s));
  c->stats.host_syncs += 1;
  std::vector<ahf_halo> h2(halos, halos + n_halos);
  for (int64_t h = 0; h < n_halos; ++h) {
    h2[(size_t)h].count = r1[(size_t)h].n_bound;
    if (r1[(size_t)h].r_vir > 0.0) h2[(size_t)h].radius = r1[(size_t)h].r_vir;
  }
  // the second pass: records, bound lists, phi and rows; removed_iter stays
  ahf_particles p2 = *p;
  return unbind_pass(c, &p2, h2.data(), n_halos, members, &p1, out, bound_idx, phi, nullptr, s, n_bins,
                     r_min_frac, prof);
}

int hier_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos, const int64_t* parent,
              const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx, void* phi,
              int32_t* removed_iter, cudaStream_t s) {
  int rc = validate(p, halos, n_halos, prm, out, bound_idx);
  if (rc) return rc;
  if (n_halos > 0 && !parent) return fail(AHF_ERR_INVALID, "parent must not be NULL");
  if (prm->variant & AHF_VAR_RETRUNCATE) return fail(AHF_ERR_INVALID, "no AHF_VAR_RETRUNCATE in a hierarchy");
  std::vector<int> depth;
  if (forest_depths(parent, n_halos, depth)) return fail(AHF_ERR_INVALID, "parent indices must form a forest");
  int max_depth = 0;
  for (int d : depth) max_depth = std::max(max_depth, d);
  if (n_halos == 0 || max_depth == 0)
    return unbind_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter, s);
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  if ((rc = validate_slots(halos, n_halos, n_slots, member_idx != nullptr))) return rc;
  // scratch outside the workspace (the levels' unbinding calls lay that out anew)
  Bump sz{nullptr, 0, 0};
  auto layout = [&](Bump& B, HierLaunch* L, int** lvl, int** anc) {
    long long* owner = B.take<long long>((size_t)std::max<int64_t>(p->n, 1));
    long long* mem = B.take<long long>((size_t)std::max<int64_t>(n_slots, 1));
    long long* cmap = B.take<long long>((size_t)std::max<int64_t>(n_slots, 1));
    int* rem = B.take<int>((size_t)std::max<int64_t>(n_slots, 1));
    ahf_result* rl = B.take<ahf_result>((size_t)n_halos);
    ahf_halo* hd = B.take<ahf_halo>((size_t)n_halos);
    int* lv = B.take<int>((size_t)n_halos);
    int* an = B.take<int>((size_t)n_halos);
    long long* kept = B.take<long long>((size_t)n_halos);
    if (L) {
      L->owner = owner; L->members = mem; L->cand_map = cmap; L->rem_level = rem; L->res_level = rl;
      L->halos = hd; L->level = lv; L->anc = an; L->kept = kept;
      *lvl = lv; *anc = an;
    }
  };
  layout(sz, nullptr, nullptr, nullptr);
  if (sz.used + 4096 > c->hier_bytes) {
    if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
    if (c->hier) cudaFree(c->hier);
    c->hier = nullptr;
    c->hier_bytes = 0;
    if (cudaMalloc(&c->hier, sz.used + 4096) != cudaSuccess) {
      cudaGetLastError();
      return fail(AHF_ERR_NOMEM, "hierarchy scratch of %zu bytes", sz.used + 4096);
    }
    c->hier_bytes = sz.used + 4096;
  }
  Bump B{(char*)c->hier, 0, c->hier_bytes};
  HierLaunch L{};
  int* d_level = nullptr;
  int* d_anc = nullptr;
  layout(B, &L, &d_level, &d_anc);
  L.member_idx = (const long long*)member_idx;
  L.n_particles = p->n;
  L.res = out;
  L.removed_iter = removed_iter;
  L.bound_idx = (const long long*)bound_idx;
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaStreamWaitEvent(s, c->last, 0));
  if (p->n) AHF_CUDA(cudaMemsetAsync(L.owner, 0xff, sizeof(long long) * (size_t)p->n, s));
  AHF_CUDA(cudaMemcpyAsync((void*)L.halos, halos, sizeof(ahf_halo) * (size_t)n_halos, cudaMemcpyHostToDevice, s));
  std::vector<int> level, anc((size_t)n_halos);
  std::vector<long long> kept;
  std::vector<ahf_halo> lh;
  int64_t launches = 0, syncs = 0;
  for (int d = max_depth; d >= 0; --d) {
    level.clear();
    for (int64_t h = 0; h < n_halos; ++h)
      if (depth[(size_t)h] == d) level.push_back((int)h);
    if (level.empty()) continue;
    for (int64_t t = 0; t < n_halos; ++t) {
      int64_t a = t;
      while (a >= 0 && depth[(size_t)a] > d) a = parent[a];
      anc[(size_t)t] = depth[(size_t)t] > d ? (int)a : -1;
    }
    const int nl = (int)level.size();
    AHF_CUDA(cudaMemcpyAsync(d_level, level.data(), sizeof(int) * (size_t)nl, cudaMemcpyHostToDevice, s));
    AHF_CUDA(cudaMemcpyAsync(d_anc, anc.data(), sizeof(int) * (size_t)n_halos, cudaMemcpyHostToDevice, s));
    L.rank = max_depth - d;
    AHF_CUDA(launch_hier_compact(L, nl, s));
    kept.assign((size_t)nl, 0);
    AHF_CUDA(cudaMemcpyAsync(kept.data(), L.kept, sizeof(long long) * (size_t)nl, cudaMemcpyDeviceToHost, s));
    AHF_CUDA(cudaStreamSynchronize(s));
    ++syncs;
    lh.resize((size_t)nl);
    for (int i = 0; i < nl; ++i) {
      lh[(size_t)i] = halos[level[(size_t)i]];
      lh[(size_t)i].count = kept[(size_t)i];
    }
    if ((rc = unbind_impl(c, p, lh.data(), nl, (const int64_t*)L.members, prm, (ahf_result*)L.res_level, bound_idx, phi,
                          removed_iter ? (int32_t*)L.rem_level : nullptr, s)))
      return rc;
    launches += c->stats.launches;
    AHF_CUDA(launch_hier_scatter(L, nl, s));
    launches += 2;
  }
  c->stats.launches = launches;
  c->stats.host_syncs += syncs;
  return end_call(c, s);
}

// The device address of a page-locked, mapped host buffer (cudaHostAlloc,
// cudaHostRegister), or NULL for pageable memory.
void* mapped_address(const void* host) {
  if (!host) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return a.devicePointer;
}

int host_impl(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
              const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx, void* phi,
              int32_t* removed_iter, int32_t n_bins, double r_min_frac, double* prof, cudaStream_t s) {
  int rc = validate(p, halos, n_halos, prm, out, bound_idx);
  if (rc) return rc;
  int64_t n_slots = p->n;
  if (member_idx) {
    n_slots = 0;
    for (int64_t h = 0; h < n_halos; ++h) n_slots = std::max<int64_t>(n_slots, halos[h].offset + halos[h].count);
  }
  const size_t es = p->coord_type == AHF_COORD_F64 ? 8 : 4;
  const size_t n = (size_t)p->n;
  const size_t ps = prm->precision == AHF_PREC_FP64 ? 8 : 4;
  const size_t bytes = align_up(6 * n * es, 256) * 1 + align_up(p->m ? n * es : 0, 256) +
                       align_up(p->u_th ? n * es : 0, 256) +
                       align_up(member_idx ? (size_t)n_slots * 8 : 0, 256) + align_up(sizeof(ahf_result) * (size_t)n_halos, 256) +
                       align_up((size_t)n_slots * 8, 256) + align_up(phi ? (size_t)n_slots * ps : 0, 256) +
                       align_up(removed_iter ? (size_t)n_slots * 4 : 0, 256) +
                       align_up(n_bins > 0 ? (size_t)n_halos * n_bins * 32 : 0, 256) + 8 * 256 + 4096;
  if (n_bins < 0 || (n_bins > 0 && n_halos > 0 && !prof)) return fail(AHF_ERR_INVALID, "profile output missing");
  if (bytes > c->stage_bytes) {
    if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    if (cudaMalloc(&c->stage, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(AHF_ERR_NOMEM, "device staging of %zu bytes", bytes);
    }
    c->stage_bytes = bytes;
  }
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaStreamWaitEvent(s, c->last, 0));
  Bump B{c->stage, 0, c->stage_bytes};
  // AHF_OPT_HOST_DIRECT 1: each buffer used in place when it is page-locked
  // and mapped; 2: the inputs so (the kernels read each candidate once, over
  // the host link, while other haloes compute), and the bound lists, phi and
  // removal iterations pushed by each class as it finishes; otherwise staged
  // through the context's device buffer
  auto direct = [&](const void* h) -> void* { return c->host_direct ? mapped_address(h) : nullptr; };
  auto out_direct = [&](const void* h) -> void* { return c->host_direct == 1 ? mapped_address(h) : nullptr; };
  ahf_particles dp = *p;
  const void* src[8] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->m, p->u_th};
  const void** dst[8] = {&dp.x, &dp.y, &dp.z, &dp.vx, &dp.vy, &dp.vz, &dp.m, &dp.u_th};
  for (int k = 0; k < 8; ++k) {
    if (!src[k]) continue;
    char* d = B.take<char>(n * es);
    if (void* m = direct(src[k])) {
      d = (char*)m;
    } else if (n) {
      AHF_CUDA(cudaMemcpyAsync(d, src[k], n * es, cudaMemcpyHostToDevice, s));
    }
    *dst[k] = d;
  }
  int64_t* dmi = nullptr;
  if (member_idx) {
    dmi = B.take<int64_t>((size_t)n_slots);
    if (void* m = direct(member_idx)) dmi = (int64_t*)m;
    else if (n_slots) AHF_CUDA(cudaMemcpyAsync(dmi, member_idx, (size_t)n_slots * 8, cudaMemcpyHostToDevice, s));
  }
  // outputs: in place when mapped (mode 1), else copied back after the kernels
  // or pushed by the classes (mode 2)
  void* m_out = n_halos ? out_direct(out) : nullptr;
  void* m_bi = n_slots ? out_direct(bound_idx) : nullptr;
  void* m_phi = (phi && n_slots) ? out_direct(phi) : nullptr;
  void* m_ri = (removed_iter && n_slots) ? out_direct(removed_iter) : nullptr;
  void* m_prof = (n_bins > 0 && n_halos) ? out_direct(prof) : nullptr;
  ahf_result* dout = B.take<ahf_result>((size_t)n_halos);
  int64_t* dbi = B.take<int64_t>((size_t)std::max<int64_t>(n_slots, 1));
  void* dphi = phi ? (void*)B.take<char>((size_t)std::max<int64_t>(n_slots, 1) * ps) : nullptr;
  int32_t* dri = removed_iter ? B.take<int32_t>((size_t)std::max<int64_t>(n_slots, 1)) : nullptr;
  double* dprof = n_bins > 0 ? B.take<double>((size_t)n_halos * n_bins * 4 + 1) : nullptr;
  if (m_out) dout = (ahf_result*)m_out;
  if (m_bi) dbi = (int64_t*)m_bi;
  if (m_phi) dphi = m_phi;
  if (m_ri) dri = (int32_t*)m_ri;
  if (m_prof) dprof = (double*)m_prof;
  // mode 2: the slot outputs go out per class when every one of them is
  // page-locked (not with the two-pass truncation variant, whose first pass
  // is overwritten)
  HostPush hp{};
  bool pushing = c->host_direct == 2 && n_slots > 0 && !(prm->variant & AHF_VAR_RETRUNCATE) &&
                 mapped_address(bound_idx) && (!phi || mapped_address(phi)) &&
                 (!removed_iter || mapped_address(removed_iter));
  if (pushing) {
    hp.res = dout;
    hp.bi = (const long long*)dbi;
    hp.h_bi = (long long*)mapped_address(bound_idx);
    hp.phi = (const char*)dphi;
    hp.h_phi = phi ? (char*)mapped_address(phi) : nullptr;
    hp.phi_es = (int)ps;
    hp.ri = dri;
    hp.h_ri = removed_iter ? (int*)mapped_address(removed_iter) : nullptr;
  }
  if ((rc = unbind_impl(c, &dp, halos, n_halos, dmi, prm, dout, dbi, dphi, dri, s, n_bins, r_min_frac,
                        n_bins > 0 ? dprof : nullptr, pushing ? &hp : nullptr)))
    return rc;
  if (n_halos && !m_out)
    AHF_CUDA(cudaMemcpyAsync(out, dout, sizeof(ahf_result) * (size_t)n_halos, cudaMemcpyDeviceToHost, s));
  if (n_bins > 0 && n_halos && !m_prof)
    AHF_CUDA(cudaMemcpyAsync(prof, dprof, sizeof(double) * (size_t)n_halos * n_bins * 4, cudaMemcpyDeviceToHost, s));
  if (n_slots && !pushing) {
    if (!m_bi) AHF_CUDA(cudaMemcpyAsync(bound_idx, dbi, (size_t)n_slots * 8, cudaMemcpyDeviceToHost, s));
    if (phi && !m_phi) AHF_CUDA(cudaMemcpyAsync(phi, dphi, (size_t)n_slots * ps, cudaMemcpyDeviceToHost, s));
    if (removed_iter && !m_ri)
      AHF_CUDA(cudaMemcpyAsync(removed_iter, dri, (size_t)n_slots * 4, cudaMemcpyDeviceToHost, s));
  }
  AHF_CUDA(cudaEventRecord(c->last, s));
  AHF_CUDA(cudaStreamSynchronize(s));
  return AHF_OK;
}

}  // namespace

extern "C" {

int ahf_version(void) { return 100; }

const char* ahf_last_error(void) { return g_last_ptr; }

const char* ahf_build_id(void) { return AHF_BUILD_ID; }

namespace {

// The device's name with every character outside [A-Za-z0-9._-] as '_'.
void device_key(int device, char* out, size_t cap) {
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof prop);
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    std::snprintf(out, cap, "unknown");
    return;
  }
  size_t k = 0;
  for (const char* p = prop.name; *p && k + 1 < cap; ++p)
    out[k++] = (std::isalnum((unsigned char)*p) || *p == '.' || *p == '-' || *p == '_') ? *p : '_';
  out[k] = 0;
}

// Tuned options from the file named by the environment variable AHF_TUNING
// (lines "device <key>", "build <id>", "option <number> <value>"; '#'
// comments).  The options are applied only when the device key and the
// build id match this device and this library; otherwise the file is
// ignored.  A file that does not parse is an error.
int apply_tuning(ahf_ctx* c) {
  const char* path = std::getenv("AHF_TUNING");
  if (!path || !*path) return AHF_OK;
  FILE* f = std::fopen(path, "r");
  if (!f) return AHF_OK;                     // no tuning yet
  char key[256];
  device_key(c->device, key, sizeof key);
  char line[512], dev[256] = {}, build[256] = {};
  std::vector<std::pair<int, long long>> opts;
  int rc = AHF_OK;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int opt = 0;
    long long val = 0;
    char word[256];
    if (std::sscanf(line, "device %255s", word) == 1) std::snprintf(dev, sizeof dev, "%s", word);
    else if (std::sscanf(line, "build %255s", word) == 1) std::snprintf(build, sizeof build, "%s", word);
    else if (std::sscanf(line, "option %d %lld", &opt, &val) == 2) opts.emplace_back(opt, val);
    else if (std::sscanf(line, "%255s", word) == 1 && word[0] != '#') {
      rc = fail(AHF_ERR_INVALID, "tuning file %s: cannot read '%s'", path, word);
      break;
    }
  }
  std::fclose(f);
  if (rc != AHF_OK) return rc;
  if (std::strcmp(dev, key) != 0 || std::strcmp(build, AHF_BUILD_ID) != 0) return AHF_OK;
  for (const auto& o : opts)
    if ((rc = ahf_set_option(c, o.first, o.second)) != AHF_OK) return rc;
  std::snprintf(c->tuning, sizeof c->tuning, "%s", path);
  return AHF_OK;
}

}  // namespace

int ahf_create(ahf_ctx** ctx, int device) {
  if (!ctx) return fail(AHF_ERR_INVALID, "ctx is NULL");
  *ctx = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return fail(AHF_ERR_INVALID, "no CUDA device %d", device);
  }
  ahf_ctx* c = new (std::nothrow) ahf_ctx();
  if (!c) return fail(AHF_ERR_NOMEM, "context allocation");
  c->device = device;
  int rc = AHF_OK;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = fail(AHF_ERR_CUDA, "cudaSetDevice(%d)", device); break; }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->err_dev, sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_NOMEM, "error word"); break; }
    if (cudaMemset(c->err_dev, 0, sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_CUDA, "memset"); break; }
    if (cudaMallocHost(&c->err_host, sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_NOMEM, "pinned word"); break; }
    if (cudaEventCreateWithFlags(&c->last, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) {
      rc = fail(AHF_ERR_CUDA, "event");
      break;
    }
    if (cudaMallocHost(&c->flag_host, 16 * sizeof(int)) != cudaSuccess) { rc = fail(AHF_ERR_NOMEM, "pinned flags"); break; }
    if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(AHF_ERR_CUDA, "capture stream");
      break;
    }
    for (int k = 0; k < NV && rc == AHF_OK; ++k) {
      if (cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->join[k], cudaEventDisableTiming) != cudaSuccess)
        rc = fail(AHF_ERR_CUDA, "side stream");
    }
    for (int k = 0; k < AHF_N_PHASES && rc == AHF_OK; ++k) {
      if (cudaEventCreate(&c->ev0[k]) != cudaSuccess || cudaEventCreate(&c->ev1[k]) != cudaSuccess)
        rc = fail(AHF_ERR_CUDA, "phase events");
    }
    for (int k = 0; k < ahf_ctx::NPIN && rc == AHF_OK; ++k)
      if (cudaEventCreateWithFlags(&c->pin_ev[k], cudaEventDisableTiming) != cudaSuccess)
        rc = fail(AHF_ERR_CUDA, "staging events");
    if (rc != AHF_OK) break;
  } while (0);
  if (rc != AHF_OK) {
    cudaGetLastError();
    ahf_destroy(c);
    return rc;
  }
  if ((rc = apply_tuning(c)) != AHF_OK) {
    ahf_destroy(c);
    return rc;
  }
  *ctx = c;
  return AHF_OK;
}

int ahf_destroy(ahf_ctx* c) {
  if (!c) return AHF_OK;
  cudaSetDevice(c->device);
  if (c->last_valid) cudaEventSynchronize(c->last);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->capture) cudaStreamDestroy(c->capture);
  if (c->trace_dev) cudaFree(c->trace_dev);
  if (c->aux) cudaFree(c->aux);
  if (c->hier) cudaFree(c->hier);
  if (c->ws) cudaFree(c->ws);
  if (c->stage) cudaFree(c->stage);
  if (c->err_dev) cudaFree(c->err_dev);
  if (c->err_host) cudaFreeHost(c->err_host);
  for (int k = 0; k < ahf_ctx::NPIN; ++k) {
    if (c->pin[k]) cudaFreeHost(c->pin[k]);
    if (c->pin_ev[k]) cudaEventDestroy(c->pin_ev[k]);
  }
  if (c->last) cudaEventDestroy(c->last);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->flag_host) cudaFreeHost(c->flag_host);
  for (int k = 0; k < NV; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->join[k]) cudaEventDestroy(c->join[k]);
  }
  for (int k = 0; k < AHF_N_PHASES; ++k) {
    if (c->ev0[k]) cudaEventDestroy(c->ev0[k]);
    if (c->ev1[k]) cudaEventDestroy(c->ev1[k]);
  }
  delete c;
  return AHF_OK;
}

int ahf_set_option(ahf_ctx* c, int option, int64_t value) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  switch (option) {
    case AHF_OPT_ONCHIP_MAX:
      if (value < 0 || value > variant_capacity(NV - 1)) return fail(AHF_ERR_INVALID, "onchip max out of range");
      c->onchip_max = value;
      return AHF_OK;
    case AHF_OPT_WAIT_LIMIT:
      if (value < 0) return fail(AHF_ERR_INVALID, "wait limit < 0");
      c->wait_limit = value;
      return AHF_OK;
    case AHF_OPT_TIMING:
      if (value != 0 && value != 1) return fail(AHF_ERR_INVALID, "timing is 0 or 1");
      c->timing = value == 1;
      return AHF_OK;
    case AHF_OPT_HOST_DIRECT:
      if (value < 0 || value > 2) return fail(AHF_ERR_INVALID, "host_direct is 0, 1 or 2");
      c->host_direct = (int)value;
      return AHF_OK;
    case AHF_OPT_GRAPHS:
      if (value != 0 && value != 1) return fail(AHF_ERR_INVALID, "graphs is 0 or 1");
      c->graphs = value == 1;
      return AHF_OK;
    case AHF_OPT_TRACE:
      if (value != 0 && value != 1) return fail(AHF_ERR_INVALID, "trace is 0 or 1");
      c->trace = value == 1;
      return AHF_OK;
    case AHF_OPT_SERIAL:
      if (value != 0 && value != 1) return fail(AHF_ERR_INVALID, "serial is 0 or 1");
      c->serial = value == 1;
      return AHF_OK;
    case AHF_OPT_PROMOTE:
      if (value != 0 && value != 1) return fail(AHF_ERR_INVALID, "promote is 0 or 1");
      c->promote = value == 1;
      return AHF_OK;
    case AHF_OPT_PASS_CHUNK:
      if (value < 1 || value > 64) return fail(AHF_ERR_INVALID, "pass chunk must be in [1, 64]");
      c->pass_chunk = (int)value;
      return AHF_OK;
    case AHF_OPT_WORKSPACE_CAP:
      if (value < 0) return fail(AHF_ERR_INVALID, "workspace cap < 0");
      c->ws_cap = value;
      return AHF_OK;
    default:
      if (option >= AHF_OPT_CLASS_CUT && option < AHF_OPT_CLASS_CUT + NV) {
        const int v = option - AHF_OPT_CLASS_CUT;
        if (value < 0 || value > variant_capacity(v))
          return fail(AHF_ERR_INVALID, "class cut of variant %d must be in [0, %d]", v, variant_capacity(v));
        c->class_cut[v] = value;
        return AHF_OK;
      }
      return fail(AHF_ERR_INVALID, "unknown option %d", option);
  }
}

int ahf_get_option(ahf_ctx* c, int option, int64_t* value) {
  if (!c || !value) return fail(AHF_ERR_INVALID, "NULL argument");
  switch (option) {
    case AHF_OPT_ONCHIP_MAX: *value = c->onchip_max; return AHF_OK;
    case AHF_OPT_WAIT_LIMIT: *value = c->wait_limit; return AHF_OK;
    case AHF_OPT_TIMING: *value = c->timing ? 1 : 0; return AHF_OK;
    case AHF_OPT_HOST_DIRECT: *value = c->host_direct; return AHF_OK;
    case AHF_OPT_GRAPHS: *value = c->graphs ? 1 : 0; return AHF_OK;
    case AHF_OPT_TRACE: *value = c->trace ? 1 : 0; return AHF_OK;
    case AHF_OPT_SERIAL: *value = c->serial ? 1 : 0; return AHF_OK;
    case AHF_OPT_PROMOTE: *value = c->promote ? 1 : 0; return AHF_OK;
    case AHF_OPT_PASS_CHUNK: *value = c->pass_chunk; return AHF_OK;
    case AHF_OPT_WORKSPACE_CAP: *value = c->ws_cap; return AHF_OK;
    default:
      if (option >= AHF_OPT_CLASS_CUT && option < AHF_OPT_CLASS_CUT + NV) {
        const int v = option - AHF_OPT_CLASS_CUT;
        *value = c->class_cut[v] >= 0 ? c->class_cut[v] : variant_capacity(v);
        return AHF_OK;
      }
      return fail(AHF_ERR_INVALID, "unknown option %d", option);
  }
}

int ahf_sync(ahf_ctx* c) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  AHF_CUDA(cudaMemcpy(c->err_host, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  const int e = *c->err_host;
  if (e) AHF_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
  if (e & ERR_TIMEOUT) return fail(AHF_ERR_TIMEOUT, "a multi-CTA pass gave up waiting for a tensor copy");
  if (e & ERR_BAD_INDEX) return fail(AHF_ERR_INVALID, "a member index was out of range");
  if (e & ERR_CAPACITY) return fail(AHF_ERR_INVALID, "a halo exceeded its size class");
  if (e & ERR_ID_RANGE) return fail(AHF_ERR_INVALID, "a catalogue particle id was out of range");
  if (e & ERR_SHARED_ID) return fail(AHF_ERR_INVALID, "a particle id is in two haloes of the second catalogue");
  if (e & ERR_MATCH_TABLE) return fail(AHF_ERR_INVALID, "a halo met more than 2048 haloes of the second catalogue");
  return AHF_OK;
}

int ahf_unbind_batch(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                     const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx,
                     void* phi, int32_t* removed_iter, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return unbind_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter,
                     (cudaStream_t)stream);
}

}  // extern "C"

extern "C" {

int ahf_unbind_batch_host(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                          const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx,
                          void* phi, int32_t* removed_iter, int32_t n_bins, double r_min_frac, double* prof,
                          void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return host_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter, n_bins, r_min_frac,
                   prof, (cudaStream_t)stream);
}

int ahf_unbind_hierarchy(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                         const int64_t* parent, const int64_t* member_idx, const ahf_params* prm, ahf_result* out,
                         int64_t* bound_idx, void* phi, int32_t* removed_iter, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return hier_impl(c, p, halos, n_halos, parent, member_idx, prm, out, bound_idx, phi, removed_iter,
                   (cudaStream_t)stream);
}

int ahf_halo_properties(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                        const int64_t* member_idx, const ahf_params* prm, const ahf_result* res,
                        const int64_t* bound_idx, const void* phi, double* props, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return props_impl(c, p, halos, n_halos, member_idx, prm, res, bound_idx, phi, props, (cudaStream_t)stream);
}

int ahf_match_catalogs(ahf_ctx* c, int64_t n_ids, const int64_t* ids_a, const int64_t* off_a, const int64_t* cnt_a,
                       int64_t n_a, const int64_t* ids_b, const int64_t* off_b, const int64_t* cnt_b, int64_t n_b,
                       int64_t* best, int64_t* shared, double* xi, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return match_impl(c, n_ids, ids_a, off_a, cnt_a, n_a, ids_b, off_b, cnt_b, n_b, best, shared, xi,
                    (cudaStream_t)stream);
}

int ahf_get_trace(ahf_ctx* c, int64_t* host, int64_t n_halos) {
  if (!c || !host) return fail(AHF_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> g(c->mu);
  if (c->trace_n < 0) return fail(AHF_ERR_INVALID, "no traced call (AHF_OPT_TRACE was off)");
  if (n_halos != c->trace_n)
    return fail(AHF_ERR_INVALID, "n_halos %lld differs from the traced call's %lld", (long long)n_halos,
                (long long)c->trace_n);
  AHF_CUDA(cudaSetDevice(c->device));
  if (c->last_valid) AHF_CUDA(cudaEventSynchronize(c->last));
  if (n_halos)
    AHF_CUDA(cudaMemcpy(host, c->trace_dev, sizeof(long long) * AHF_TRACE_FIELDS * (size_t)n_halos,
                        cudaMemcpyDeviceToHost));
  return AHF_OK;
}

int ahf_get_stats(ahf_ctx* c, ahf_stats* out) {
  if (!c || !out) return fail(AHF_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> g(c->mu);
  if (c->timing) {
    AHF_CUDA(cudaSetDevice(c->device));
    for (int k = 0; k < AHF_N_PHASES; ++k) {
      if (!c->phase_used[k]) continue;
      AHF_CUDA(cudaEventSynchronize(c->ev1[k]));
      float ms = 0.0f;
      AHF_CUDA(cudaEventElapsedTime(&ms, c->ev0[k], c->ev1[k]));
      c->stats.phase_ms[k] = ms;
    }
  }
  *out = c->stats;
  return AHF_OK;
}

int ahf_unbind_plain(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                     const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx,
                     void* phi, int32_t* removed_iter, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return plain_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter, (cudaStream_t)stream);
}

int ahf_unbind_profile_batch(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                             const int64_t* member_idx, const ahf_params* prm, ahf_result* out, int64_t* bound_idx,
                             void* phi, int32_t* removed_iter, int32_t n_bins, double r_min_frac, double* prof,
                             void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  if (n_halos > 0 && !prof) return fail(AHF_ERR_INVALID, "prof must not be NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return unbind_impl(c, p, halos, n_halos, member_idx, prm, out, bound_idx, phi, removed_iter, (cudaStream_t)stream,
                     n_bins, r_min_frac, n_halos > 0 ? prof : nullptr);
}

int ahf_profile_batch(ahf_ctx* c, const ahf_particles* p, const ahf_halo* halos, int64_t n_halos,
                      const int64_t* member_idx, const ahf_params* prm, const ahf_result* res,
                      const int64_t* bound_idx, int32_t n_bins, double r_min_frac, double* prof, void* stream) {
  if (!c) return fail(AHF_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::mutex> g(c->mu);
  return profile_impl(c, p, halos, n_halos, member_idx, prm, res, bound_idx, n_bins, r_min_frac, prof,
                      (cudaStream_t)stream);
}

}  // extern "C"
